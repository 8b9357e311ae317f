"""Thin ctypes binding of the C ABI in include/fwi.h (argument marshalling only: every step
of the forward, adjoint and gradient computation runs in the CUDA library).

Bulk arrays may be torch tensors (CUDA or CPU) or numpy arrays; the library itself tells
device from host pointers. The library must have been built (``build()`` in this package);
there is no fallback: a missing library raises.
"""
import ctypes
import os

import numpy as np

from . import _build

FWI_EINVAL, FWI_ENOMEM, FWI_ERANGE, FWI_ECUDA, FWI_ETIMEDOUT = -22, -12, -34, -5, -110


class FwiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fwi error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("k", ctypes.c_int), ("dt", ctypes.c_double),
                ("cfl_factor", ctypes.c_double), ("nsteps", ctypes.c_int),
                ("box_lo", ctypes.c_double * 3), ("box_hi", ctypes.c_double * 3),
                ("layer_faces", ctypes.c_int), ("layer_width", ctypes.c_double),
                ("sigma_max", ctypes.c_double), ("absorbing", ctypes.c_int),
                ("ckpt_stride", ctypes.c_int), ("water_speed", ctypes.c_double),
                ("layout", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("grad_stride", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def library_path():
    return _build.LIB


def load():
    """Load libfwi_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run build())")
    lib = ctypes.CDLL(path)
    sig = {
        "fwi_mesh_upload": (ctypes.c_int, [_P, _I64, _P, _I64, ctypes.POINTER(Params), ctypes.POINTER(_P)]),
        "fwi_mesh_prepare_host": (ctypes.c_int, [_P, _I64, _P, _I64, ctypes.POINTER(Params), ctypes.POINTER(_P)]),
        "fwi_mesh_host_arrays": (ctypes.c_int, [_P, _P, _P, _P, _P]),
        "fwi_num_dofs": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
        "fwi_dof_coords": (ctypes.c_int, [_P, _P]),
        "fwi_element": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), _P, _P, _P]),
        "fwi_set_velocity": (ctypes.c_int, [_P, _P]),
        "fwi_locate": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
        "fwi_reference_element": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                 _P, _P, _P, ctypes.POINTER(ctypes.c_int)]),
        "fwi_get_dt": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
        "fwi_reference_element_f32": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P]),
        "fwi_batch_create": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, _P, ctypes.POINTER(_P)]),
        "fwi_forward_shot": (ctypes.c_int, [_P, _P, _P, _P]),
        "fwi_adjoint_shot": (ctypes.c_int, [_P, _P, _P]),
        "fwi_forward_shot_noalloc": (ctypes.c_int, [_P, _P, _P, _P]),
        "fwi_adjoint_misfit": (ctypes.c_int, [_P, _P, _P]),
        "fwi_gradient": (ctypes.c_int, [_P, _P, _P, _P]),
        "fwi_gradient_lanes": (ctypes.c_int, [_P, _P, _P, _P]),
        "fwi_forward_segment": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint32, _P, _P, _P]),
        "fwi_batch_free": (ctypes.c_int, [_P]),
        "fwi_batch_set_sources": (ctypes.c_int, [_P, _P]),
        "fwi_batch_bytes": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_I64)]),
        "fwi_gradient_raw": (ctypes.c_int, [_P, _P, _P, _P]),
        "fwi_profile": (ctypes.c_int, [_P, ctypes.c_int]),
        "fwi_batch_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_int]),
        "fwi_batch_set_gradient_lanes": (ctypes.c_int, [_P, ctypes.c_int]),
        "fwi_batch_set_gradient_store": (ctypes.c_int, [_P, ctypes.c_int]),
        "fwi_profile_read": (ctypes.c_int, [_P, _P, _P]),
        "fwi_mesh_free": (ctypes.c_int, [_P]),
        "fwi_last_error": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int]),
        "fwi_launch_count": (ctypes.c_int64, []),
        "fwi_fp32_peak": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return [n for n in dir(load()) if n.startswith("fwi_")]


def _check(rc):
    if rc != 0:
        buf = ctypes.create_string_buffer(512)
        _lib.fwi_last_error(buf, 512)
        raise FwiError(rc, buf.value.decode(errors="replace"))


def _ptr(x):
    """data pointer of a torch tensor or numpy array (must be contiguous)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data)


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def reference_element(dim, k):
    """(nodes [n][dim], weights [n], dhat [dim][n][n], exact degree) of the library's own
    KMV tabulation (host only, no GPU needed)."""
    lib = load()
    n = ctypes.c_int()
    deg = ctypes.c_int()
    _check(lib.fwi_reference_element(dim, k, ctypes.byref(n), None, None, None, ctypes.byref(deg)))
    nn = n.value
    xh = np.zeros((nn, dim))
    w = np.zeros(nn)
    dh = np.zeros((dim, nn, nn))
    _check(lib.fwi_reference_element(dim, k, ctypes.byref(n), _ptr(xh), _ptr(w), _ptr(dh),
                                     ctypes.byref(deg)))
    return xh, w, dh, deg.value


def reference_element_f32(dim, k):
    """(dhat [dim][n][n], w [n]) as the FP32 tables the kernels use (host only)."""
    xh, _, _, _ = reference_element(dim, k)
    n = xh.shape[0]
    dh = np.zeros((dim, n, n), dtype=np.float32)
    w = np.zeros(n, dtype=np.float32)
    _check(load().fwi_reference_element_f32(dim, k, _ptr(dh), _ptr(w)))
    return dh, w


def fp32_peak():
    """(measured FP32 FMA TFLOP/s of the current device, its SM count)."""
    t = ctypes.c_double()
    n = ctypes.c_int()
    _check(load().fwi_fp32_peak(ctypes.byref(t), ctypes.byref(n)))
    return t.value, n.value


def launch_count():
    return int(load().fwi_launch_count())


class Mesh:
    """A mesh resident on the current CUDA device (fwi_mesh_upload)."""

    def __init__(self, verts, cells, k, nsteps, dt=0.0, cfl_factor=0.9, box=None, layer_faces=0,
                 layer_width=0.0, sigma_max=0.0, absorbing=False, ckpt_stride=50, water_speed=0.0,
                 host_only=False, layout=0, tensor_cores=0, grad_stride=1):
        lib = load()
        verts = np.ascontiguousarray(verts, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        p = Params()
        p.dim = verts.shape[1]
        p.k = int(k)
        p.dt = float(dt)
        p.cfl_factor = float(cfl_factor)
        p.nsteps = int(nsteps)
        if box is not None:
            for i, (lo, hi) in enumerate(box):
                p.box_lo[i] = lo
                p.box_hi[i] = hi
        p.layer_faces = int(layer_faces)
        p.layer_width = float(layer_width)
        p.sigma_max = float(sigma_max)
        p.absorbing = int(bool(absorbing))
        p.ckpt_stride = int(ckpt_stride)
        p.water_speed = float(water_speed)
        p.layout = int(layout)
        p.tensor_cores = int(tensor_cores)
        p.grad_stride = int(grad_stride)
        self.params = p
        self.dim = p.dim
        h = ctypes.c_void_p()
        fn = lib.fwi_mesh_prepare_host if host_only else lib.fwi_mesh_upload
        _check(fn(_ptr(verts), verts.shape[0], _ptr(cells), cells.shape[0], ctypes.byref(p),
                  ctypes.byref(h)))
        self.E = cells.shape[0]
        self._h = h
        n = ctypes.c_int64()
        _check(lib.fwi_num_dofs(h, ctypes.byref(n)))
        self.N = n.value

    def dof_coords(self):
        out = np.zeros((self.N, self.dim))
        _check(_lib.fwi_dof_coords(self._h, _ptr(out)))
        return out

    def element(self):
        n = ctypes.c_int()
        _check(_lib.fwi_element(self._h, ctypes.byref(n), None, None, None))
        nn = n.value
        xh = np.zeros((nn, self.dim))
        w = np.zeros(nn)
        dh = np.zeros((self.dim, nn, nn))
        _check(_lib.fwi_element(self._h, ctypes.byref(n), _ptr(xh), _ptr(w), _ptr(dh)))
        return xh, w, dh

    def host_arrays(self):
        """(conn [E][n], mass [N], boundary mass [N], sigma [N][dim]) as prepared on the host."""
        xh, _, _ = self.element()
        n = xh.shape[0]
        conn = np.zeros((self.E, n), dtype=np.int32)
        M = np.zeros(self.N)
        Mb = np.zeros(self.N)
        sig = np.zeros((self.N, self.dim))
        _check(_lib.fwi_mesh_host_arrays(self._h, _ptr(conn), _ptr(M), _ptr(Mb), _ptr(sig)))
        return conn, M, Mb, sig

    def locate(self, pts):
        """(element index in the library's order [npts], reference coordinates [npts][dim])
        of each point; raises FwiError(FWI_EINVAL) for a point outside the mesh."""
        pts = np.ascontiguousarray(np.atleast_2d(pts), dtype=np.float64)
        el = np.zeros(pts.shape[0], dtype=np.int32)
        xh = np.zeros((pts.shape[0], self.dim))
        _check(_lib.fwi_locate(self._h, _ptr(pts), pts.shape[0], _ptr(el), _ptr(xh)))
        return el, xh

    def set_velocity(self, c):
        c = np.ascontiguousarray(c, dtype=np.float64)
        if c.shape != (self.N,):
            raise ValueError("velocity must have one value per DoF")
        _check(_lib.fwi_set_velocity(self._h, _ptr(c)))

    @property
    def dt(self):
        v = ctypes.c_double()
        _check(_lib.fwi_get_dt(self._h, ctypes.byref(v)))
        return v.value

    @property
    def nsteps(self):
        return self.params.nsteps

    def batch_bytes(self, nshots, nrec):
        """Device bytes a batch of nshots shots and nrec receivers would allocate."""
        v = ctypes.c_int64()
        _check(_lib.fwi_batch_bytes(self._h, int(nshots), int(nrec), ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.fwi_mesh_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """S shots over one mesh with a shared receiver spread (fwi_batch_create)."""

    def __init__(self, mesh, src, rec):
        src = np.ascontiguousarray(np.atleast_2d(src), dtype=np.float64)
        rec = np.ascontiguousarray(np.atleast_2d(rec), dtype=np.float64)
        self.mesh = mesh
        self.S = src.shape[0]
        self.R = rec.shape[0]
        h = ctypes.c_void_p()
        _check(_lib.fwi_batch_create(mesh._h, self.S, _ptr(src), self.R, _ptr(rec), ctypes.byref(h)))
        self._h = h

    def forward(self, wavelet, rec_out, stream=None):
        """wavelet [S][Nt] float32, rec_out [S][Nt+1][R] float32 (host or device)."""
        _check(_lib.fwi_forward_shot(self._h, _ptr(wavelet), _ptr(rec_out), _stream_ptr(stream)))

    def forward_noalloc(self, wavelet, rec_out, stream=None):
        """fwi_forward_shot_noalloc: the forward solve with no device allocation (device
        pointers only; see include/fwi.h for the shared static scratch and its limits)."""
        _check(_lib.fwi_forward_shot_noalloc(self._h, _ptr(wavelet), _ptr(rec_out),
                                             _stream_ptr(stream)))

    def adjoint(self, residual, stream=None):
        """residual [S][Nt+1][R] float32 = d - dtilde (host or device)."""
        _check(_lib.fwi_adjoint_shot(self._h, _ptr(residual), _stream_ptr(stream)))

    def adjoint_misfit(self, observed, stream=None):
        """observed [S][Nt+1][R] float32 (host or device); residual formed on the device."""
        _check(_lib.fwi_adjoint_misfit(self._h, _ptr(observed), _stream_ptr(stream)))

    def set_sources(self, src):
        """Move the batch's S sources (host coordinates) without reallocating."""
        src = np.ascontiguousarray(np.atleast_2d(src), dtype=np.float64)
        if src.shape[0] != self.S:
            raise ValueError("set_sources needs exactly S positions")
        _check(_lib.fwi_batch_set_sources(self._h, _ptr(src)))

    def gradient_raw(self, out, stream=None):
        """out [N] float64 = dJ/dc (masked, no mass solve); returns the misfit J."""
        J = ctypes.c_double()
        _check(_lib.fwi_gradient_raw(self._h, _ptr(out), ctypes.byref(J), _stream_ptr(stream)))
        return J.value

    def gradient(self, out, stream=None):
        """out [N] float64 (host or device); returns the misfit J."""
        J = ctypes.c_double()
        _check(_lib.fwi_gradient(self._h, _ptr(out), ctypes.byref(J), _stream_ptr(stream)))
        return J.value

    def forward_segment(self, nseg, reset_mask, wavelet, rec_out=None, stream=None):
        """Advance every lane by nseg steps (lanes in reset_mask start a new shot first);
        wavelet [S][nseg], rec_out [S][nseg+1][R] (host or device)."""
        _check(_lib.fwi_forward_segment(self._h, int(nseg), ctypes.c_uint32(int(reset_mask)),
                                        _ptr(wavelet), _ptr(rec_out), _stream_ptr(stream)))

    def set_gradient_lanes(self, per_shot=True):
        """Keep each shot's gradient apart in the next adjoint calls (for gradient_lanes)."""
        _check(_lib.fwi_batch_set_gradient_lanes(self._h, int(bool(per_shot))))

    def set_gradient_store(self, on=True):
        """Store the forward field's gradients during the recompute (faster gradient steps,
        more device memory; see fwi_batch_set_gradient_store)."""
        _check(_lib.fwi_batch_set_gradient_store(self._h, int(bool(on))))

    def gradient_lanes(self, out, stream=None):
        """out [S][N] float64 (host or device) = each shot's own gradient; returns the S
        misfits J_s as a float64 array."""
        J = np.zeros(self.S)
        _check(_lib.fwi_gradient_lanes(self._h, _ptr(out), _ptr(J), _stream_ptr(stream)))
        return J

    def set_wait_limit(self, polls):
        """Polls per bounded tensor-core wait (testing aid; -1 restores the default)."""
        _check(_lib.fwi_batch_set_wait_limit(self._h, int(polls)))

    def profile(self, enable=True):
        _check(_lib.fwi_profile(self._h, int(bool(enable))))

    def profile_read(self):
        """{'fwd_elem_ms', 'fwd_node_ms', 'adj_elem_ms', 'adj_node_ms', 'fwd_steps',
        'adj_steps'} since the last read."""
        ms = np.zeros(4)
        steps = np.zeros(2, dtype=np.int64)
        _check(_lib.fwi_profile_read(self._h, _ptr(ms), _ptr(steps)))
        return dict(fwd_elem_ms=ms[0], fwd_node_ms=ms[1], adj_elem_ms=ms[2], adj_node_ms=ms[3],
                    fwd_steps=int(steps[0]), adj_steps=int(steps[1]))

    def close(self):
        if getattr(self, "_h", None):
            _lib.fwi_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
