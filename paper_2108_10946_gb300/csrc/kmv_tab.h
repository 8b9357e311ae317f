// Reference-element tabulation of the KMV mass-lumped simplices (host, FP64 output,
// long double internally). Section 3.2 and Section 4.2 of the paper: P_k enriched with
// bubbles, nodes that double as the points of the lumping quadrature, nodal basis.
#pragma once
#include <string>
#include <vector>

namespace kmvtab {

struct Term {
  int e[3];
  long double c;
};
using Poly = std::vector<Term>;

// Node entity classes, used by the DoF numbering.
enum Entity { VERTEX = 0, EDGE = 1, FACE = 2, INTERIOR = 3 };

struct Element {
  int dim = 0, k = 0, n = 0;
  int exact_degree = -1;
  std::vector<double> bary;   // [n][dim+1]
  std::vector<double> xhat;   // [n][dim]
  std::vector<double> w;      // [n], sums to 1/dim!
  std::vector<double> dhat;   // [dim][n][n]: d phi_j / d xhat_d at node q
  std::vector<int> entity;    // [n] Entity
  std::vector<int> ent_verts; // [n][3] local vertices spanning the node's entity (-1 pad)
  std::vector<int> ent_rank;  // [n] order of the node inside its entity (see kmv_tab.cpp)
  std::vector<std::vector<int>> facet_nodes;      // [dim+1]: nodes on facet opposite vertex i
  std::vector<std::vector<double>> facet_weights; // lumped facet rule (sums to 1 or 1/2)
  std::vector<Poly> space;
  std::vector<long double> coef; // [n_space][n]: phi_j = sum_m space_m * coef[m][j]
  void basis(const double* x, double* phi) const;  // phi[n] at reference point x
};

// Builds KMVktri (dim 2, k 2..5) or KMVktet (dim 3, k 2..3). Returns false with a message.
bool build(int dim, int k, Element& out, std::string& err);

// FP32 tables for the kernels: dhat32[dim][n][n] and w32[n], rounded so that the identities
// every derivative row and the weights satisfy exactly in FP64 still hold as closely as FP32
// values allow: each row of dhat differentiates the polynomials of degree <= 2 at its node,
// and the weights integrate degree <= 1 (see kmv_tab.cpp).
void fp32_tables(const Element& el, std::vector<float>& dhat32, std::vector<float>& w32);

}  // namespace kmvtab
