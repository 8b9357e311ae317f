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
