"""CPU-only checks of the boundary: the library builds, loads, and exports every entry
point that include/fwi.h declares; the binding refuses to run without the library."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "fwi.h")).read()
    return sorted(set(re.findall(r"\b(fwi_[a-z_]+)\s*\(", text)))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ("fwi_mesh_upload", "fwi_forward_shot", "fwi_adjoint_shot", "fwi_gradient",
              "fwi_mesh_free", "fwi_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import ctypes
    import paper_2108_10946_gb300 as pkg
    path = pkg.build()
    lib = ctypes.CDLL(path)  # loads without a GPU: no CUDA call happens at load time
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2108_10946_gb300.lib as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        L.load()


@pytest.mark.parametrize("dim,k", [(2, 2), (2, 3), (2, 4), (2, 5), (3, 2), (3, 3)])
def test_library_tabulation_matches_oracle(dim, k):
    """The library's C++ KMV tabulation and the oracle's are independent implementations of
    the same element: nodes (as a set), weights and derivative matrices must agree."""
    import numpy as np
    from oracle import kmv
    import paper_2108_10946_gb300.lib as L
    xh, w, dh, deg = L.reference_element(dim, k)
    e = kmv.kmv(dim, k)
    assert deg == e.exact_degree
    # match nodes
    perm = [int(np.argmin(np.linalg.norm(e.nodes - x, axis=1))) for x in xh]
    assert sorted(perm) == list(range(e.n))
    assert np.allclose(e.nodes[perm], xh, atol=1e-13)
    assert np.allclose(e.weights[perm], w, atol=1e-14)
    assert np.allclose(e.Dhat[:, perm][:, :, perm], dh, atol=1e-9)


@pytest.mark.parametrize("dim,layout", [(2, 1), (3, 0)])
def test_tensor_cores_refused_where_there_is_no_such_kernel(dim, layout):
    """tensor_cores = 1 asks for the tensor-core chunk kernel, which exists for triangles in
    the chunked layout only; the mesh call refuses anything else (host-only preparation, no
    GPU needed)."""
    import numpy as np
    import paper_2108_10946_gb300 as pkg
    from synth import meshes
    pkg.build()
    if dim == 2:
        V, C = meshes.structured_tri(4, 4)
    else:
        g = np.linspace(0.0, 1.0, 3)
        V, C = meshes.kuhn_tets(g, g, g)
    with pytest.raises(RuntimeError, match="tensor_cores"):
        pkg.Mesh(V, C, 2, 10, dt=1e-3, host_only=True, layout=layout, tensor_cores=1)
    m = pkg.Mesh(V, C, 2, 10, dt=1e-3, host_only=True, layout=layout, tensor_cores=0)
    assert m.N > 0
    m.close()


# ---- error paths of the boundary (host side, no GPU) -------------------------------------

def _host_mesh(V, C, k=2, **kw):
    import paper_2108_10946_gb300 as pkg
    pkg.build()
    return pkg.Mesh(V, C, k, 10, dt=1e-3, host_only=True, **kw)


def test_inverted_cell_is_refused_with_einval():
    """An element with det J <= 0 (its vertices listed clockwise) is an invalid mesh: the
    library returns FWI_EINVAL and names the element."""
    import paper_2108_10946_gb300.lib as L
    from synth import meshes
    V, C = meshes.structured_tri(4, 4)
    C = C.copy()
    C[5] = C[5][[0, 2, 1]]
    with pytest.raises(L.FwiError, match="det J") as ei:
        _host_mesh(V, C)
    assert ei.value.code == L.FWI_EINVAL


@pytest.mark.parametrize("dim", [2, 3])
def test_point_outside_the_mesh_is_refused_with_einval(dim):
    """Point location (Section 4.2) of a receiver outside the domain: FWI_EINVAL; points
    inside (including a shared vertex) are found with reference coordinates that map back
    to the point."""
    import numpy as np
    import paper_2108_10946_gb300.lib as L
    from synth import meshes
    if dim == 2:
        V, C = meshes.structured_tri(6, 6)
        inside = np.array([[0.31, 0.72], [0.5, 0.5], [0.0, 0.0]])
        outside = np.array([[0.3, 0.2], [1.2, 0.5]])
    else:
        g = np.linspace(0.0, 1.0, 4)
        V, C = meshes.kuhn_tets(g, g, g)
        inside = np.array([[0.31, 0.72, 0.4], [1 / 3, 1 / 3, 1 / 3]])
        outside = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, -0.01]])
    m = _host_mesh(V, C)
    el, xh = m.locate(inside)
    conn = m.host_arrays()[0]
    xyz = m.dof_coords()
    nv = dim + 1  # the first dim+1 local nodes of every element are its vertices
    for p in range(len(inside)):
        X = xyz[conn[el[p], :nv]]
        back = X[0] + (X[1:] - X[0]).T @ xh[p]
        assert np.allclose(back, inside[p], atol=1e-12)
    with pytest.raises(L.FwiError, match="outside the mesh") as ei:
        m.locate(outside)
    assert ei.value.code == L.FWI_EINVAL
    m.close()


def test_batch_bytes_counts_every_device_array():
    """fwi_batch_bytes, the admission test of the shot server, against the sizes of the
    arrays a batch allocates (host-only mesh, no GPU): wavefields, layer auxiliaries,
    checkpoints, the recompute ring, per-shot gradient accumulators and the signal copies."""
    import numpy as np
    from synth import meshes, signals
    V, C = meshes.structured_tri(12, 10, 1.2, 1.0, -0.1, 0.0)
    m = _host_mesh(V, C, k=3, box=[(0.0, 1.0), (-10.0, 0.9)], layer_faces=0b1011,
                   layer_width=0.1, sigma_max=signals.sigma_max(2.0, 0.1), ckpt_stride=7)
    S, R, nt = 4, 9, 10
    N = m.N
    conn = m.host_arrays()[0]
    sig = m.host_arrays()[3]
    # DoFs of damping-layer elements (an element is one when a vertex lies inside the
    # layer; the first dim + 1 local nodes are the vertices) carry the layer auxiliaries
    layer_el = np.any(np.any(sig[conn[:, :3]] > 0, axis=2), axis=1)
    Nl = len(np.unique(conn[layer_el]))
    C_ = -(-nt // 7)
    state = S * (2 * N + Nl * 2)
    floats = (3 * N * S + 3 * Nl * 2 * S + 2 * Nl * S + 2 * N * S + Nl * 2 * S + Nl * S
              + state * C_ + N * S * 7 + N * S + 2 * S * (nt + 1) * R + S * nt)
    expect = floats * 4 + 2 * N * S * 8 + m.E * 4  # per-shot gradient sums
    assert m.batch_bytes(S, R) == expect
    m.close()


@pytest.mark.parametrize("dim,k", [(2, 2), (2, 3), (2, 4), (2, 5), (3, 2), (3, 3)])
def test_fp32_tables_keep_the_polynomial_identities(dim, k):
    """The kernels' FP32 copies of Dhat and w are not nearest-rounded: every derivative row
    still differentiates the polynomials of degree <= 2 at its node to within a small
    fraction of what nearest rounding leaves (that residual is the same in every element and
    drifts the phase of long records), and the weights still sum to the reference volume.
    Each entry stays within a few FP32 spacings (of its row's largest entry) of its FP64
    value."""
    import numpy as np
    from oracle import kmv
    import paper_2108_10946_gb300.lib as L
    dh32, w32 = L.reference_element_f32(dim, k)
    xh, w64, dh64, _ = L.reference_element(dim, k)
    monos = kmv._monomials(dim, 2)
    A = np.stack([kmv.peval(kmv._mono(e), xh) for e in monos])
    near = new = 0.0
    for d in range(dim):
        for q in range(len(xh)):
            b = np.array([kmv.pgrad(kmv._mono(e), xh[q:q + 1])[0, d] for e in monos])
            near = max(near, np.abs(A @ dh64[d, q].astype(np.float32).astype(np.float64) - b).max())
            new = max(new, np.abs(A @ dh32[d, q].astype(np.float64) - b).max())
    print(f"dim {dim} k {k}: P2 residual of the FP32 rows {new:.2e} (nearest rounding {near:.2e})")
    assert new < 3e-8 and new < near / 5
    # each entry moves by at most a few spacings of the coarsest FP32 value in its row
    row_ulp = np.spacing(np.abs(dh64).max(axis=2).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(dh32.astype(np.float64) - dh64).max(axis=2) <= 4 * row_ulp)
    vol = 0.5 if dim == 2 else 1.0 / 6.0
    assert abs(np.sum(w32.astype(np.float64)) - vol) < 1e-10
    assert np.abs(w32.astype(np.float64) - w64).max() <= 4 * np.abs(w64.astype(np.float32) - w64).max() + 1e-12
