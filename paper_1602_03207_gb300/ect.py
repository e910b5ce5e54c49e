"""Thin Python binding of the C ABI in include/ect.h (argument marshalling only).

Every computation runs in libect.so.  Host arrays are numpy arrays; device
buffers are torch CUDA tensors (complex128 or complex64, contiguous) whose
data pointers are handed to the library.  There is no CPU fallback: if the
library is missing or fails to load, every entry point raises.

Each Context owns a dedicated CUDA stream; calls order themselves after the
caller's current torch stream and make it wait for the library's work, so
tensors can be used as ordinary torch tensors before and after a call.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libect.so")

ECT_OK = 0
ECT_ERR_ARG, ECT_ERR_MESH, ECT_ERR_CUDA, ECT_ERR_OOM = 1, 2, 3, 4
ECT_ERR_NOT_CONVERGED, ECT_ERR_BREAKDOWN, ECT_ERR_TIMEOUT, ECT_ERR_STATE = 5, 6, 7, 8
ECT_VACUUM, ECT_DEFECT = 0, 1
ECT_F64, ECT_F32 = 1, 2
ECT_MODE_F64, ECT_MODE_MIXED = 0, 1


def sweep_matrix(f, config):
    """Matrix index of configuration `config` at sweep frequency f (ECT_SWEEP_MATRIX)."""
    return 2 + 2 * int(f) + int(config)

_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_MESH", 3: "ERR_CUDA", 4: "ERR_OOM", 5: "ERR_NOT_CONVERGED",
          6: "ERR_BREAKDOWN", 7: "ERR_TIMEOUT", 8: "ERR_STATE"}

# every symbol include/ect.h declares
EXPORTS = ["ect_default_options", "ect_create", "ect_destroy", "ect_last_error", "ect_set_mesh",
           "ect_set_physics", "ect_assemble", "ect_precond_setup", "ect_matrix_info", "ect_matrix_copy",
           "ect_scaling_copy", "ect_spmv", "ect_precond_apply", "ect_cgs2", "ect_coil_rhs", "ect_solve",
           "ect_delta_z", "ect_impedance", "ect_autotune", "ect_set_defect", "ect_delta_z_static", "ect_set_spmm_rows", "ect_partition", "ect_set_ibc", "ect_assemble_sweep", "ect_solve_sweep", "ect_set_block_split", "ect_get_block_split",
           "ect_impedance_sweep", "ect_mlp_num_params", "ect_mlp_create",
           "ect_mlp_destroy", "ect_mlp_last_error", "ect_mlp_set_params", "ect_mlp_get_params", "ect_mlp_forward",
           "ect_mlp_gradients", "ect_mlp_train_step"]


class EctError(RuntimeError):
    def __init__(self, code, msg, stats=None):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code
        self.stats = stats


class Coil(ctypes.Structure):
    _fields_ = [("r_in", ctypes.c_double), ("r_out", ctypes.c_double), ("length", ctypes.c_double),
                ("z_offset", ctypes.c_double), ("J_e", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("mode", ctypes.c_int), ("inner_iters", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("rhs_tile", ctypes.c_int), ("timeout_s", ctypes.c_double), ("reorth", ctypes.c_int),
                ("spmm_rows", ctypes.c_int), ("x0", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("restarts", ctypes.c_int), ("relres_max", ctypes.c_double), ("ms", ctypes.c_double),
                ("launches", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load_library(path=LIB_PATH):
    """Load libect.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with __graft_entry__.build() "
                           "or python paper_1602_03207_gb300/build.py")
    L = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "ect_default_options": (None, [ctypes.POINTER(Options)]),
        "ect_create": (I, [ctypes.POINTER(P), P]),
        "ect_destroy": (None, [P]),
        "ect_last_error": (ctypes.c_char_p, [P]),
        "ect_set_mesh": (I, [P, P, I64, P, I64, P, P, P, P, P, P]),
        "ect_set_physics": (I, [P, D, D, D]),
        "ect_set_defect": (I, [P, P, P]),
        "ect_assemble": (I, [P, I, I]),
        "ect_precond_setup": (I, [P, I, I, I]),
        "ect_matrix_info": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "ect_matrix_copy": (I, [P, I, P, P, P]),
        "ect_scaling_copy": (I, [P, I, P]),
        "ect_spmv": (I, [P, I, I, P, P, I]),
        "ect_precond_apply": (I, [P, I, I, P, P, I]),
        "ect_set_spmm_rows": (I, [P, I]),
        "ect_partition": (I, [P, I64, I, P, P]),
        "ect_set_ibc": (I, [P, I, P, D, D]),
        "ect_assemble_sweep": (I, [P, P, I, I]),
        "ect_set_block_split": (I, [P, I]),
        "ect_get_block_split": (I, [P]),
        "ect_solve_sweep": (I, [P, I, P, P, I, ctypes.POINTER(Options), ctypes.POINTER(Stats)]),
        "ect_impedance_sweep": (I, [P, ctypes.POINTER(Coil), P, I, ctypes.POINTER(Options), P, ctypes.POINTER(Stats)]),
        "ect_cgs2": (I, [P, I, P, I, I64, P, P, P]),
        "ect_coil_rhs": (I, [P, ctypes.POINTER(Coil), P, I, P]),
        "ect_solve": (I, [P, I, P, P, I, ctypes.POINTER(Options), ctypes.POINTER(Stats)]),
        "ect_delta_z": (I, [P, P, P, P, P, P, P]),
        "ect_delta_z_static": (I, [P, P, P, P, P, I, P, P]),
        "ect_autotune": (I, [P, I, P, P, I, ctypes.POINTER(Options), ctypes.POINTER(Options), ctypes.POINTER(Stats)]),
        "ect_impedance": (I, [P, ctypes.POINTER(Coil), P, I, ctypes.POINTER(Options), P, ctypes.POINTER(Stats)]),
        "ect_mlp_num_params": (I, []),
        "ect_mlp_create": (I, [ctypes.POINTER(P), P, I]),
        "ect_mlp_destroy": (None, [P]),
        "ect_mlp_last_error": (ctypes.c_char_p, [P]),
        "ect_mlp_set_params": (I, [P, P]),
        "ect_mlp_get_params": (I, [P, P]),
        "ect_mlp_forward": (I, [P, P, P]),
        "ect_mlp_gradients": (I, [P, P, P, P, P]),
        "ect_mlp_train_step": (I, [P, P, P, ctypes.c_float, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def default_options(**kw):
    o = Options()
    load_library().ect_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def partition(xyz, max_block_nodes=16):
    """Recursive coordinate bisection (ect_partition): returns (new_id, block_of_new)."""
    L = load_library()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    new_id = np.empty(n, dtype=np.int32)
    blk = np.empty(n, dtype=np.int32)
    rc = L.ect_partition(_ptr(xyz), n, int(max_block_nodes), _ptr(new_id), _ptr(blk))
    if rc != 0:
        raise EctError(rc, L.ect_last_error(None).decode())
    return new_id, blk


def _ptr(a):
    """Host pointer of a contiguous numpy array (None -> NULL)."""
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _dptr(t):
    """Device pointer of a contiguous torch CUDA tensor."""
    assert t.is_cuda and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def coil(c):
    """ect_coil from an object with r_in, r_out, length, z_offset, J_e."""
    return Coil(c.r_in, c.r_out, c.length, c.z_offset, c.J_e)


class Context:
    """One ect_ctx bound to its own CUDA stream on the current device."""

    def __init__(self):
        import torch
        self._torch = torch
        self.L = load_library()
        self.stream = torch.cuda.Stream()
        h = ctypes.c_void_p()
        rc = self.L.ect_create(ctypes.byref(h), ctypes.c_void_p(self.stream.cuda_stream))
        if rc != ECT_OK:
            raise EctError(rc, self.L.ect_last_error(None).decode())
        self.h = h
        self.n_nodes = 0
        self.n_sweep = 0

    def close(self):
        if getattr(self, "h", None):
            self.L.ect_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ordering with the caller's torch stream
    def _call(self, fn, *args, stats=None):
        cur = self._torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        rc = fn(self.h, *args)
        cur.wait_stream(self.stream)
        if rc != ECT_OK:
            raise EctError(rc, self.L.ect_last_error(self.h).decode(), stats)
        return rc

    # ---- ect_set_mesh / ect_set_physics ------------------------------------
    def set_mesh(self, xyz, tets, sigma, nu, sigma_d, nu_d, block_of_node, bc_mask):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        nu = np.ascontiguousarray(nu, dtype=np.float64)
        sd = None if sigma_d is None else np.ascontiguousarray(sigma_d, dtype=np.float64)
        nd = None if nu_d is None else np.ascontiguousarray(nu_d, dtype=np.float64)
        bon = np.ascontiguousarray(block_of_node, dtype=np.int32)
        bc = np.ascontiguousarray(bc_mask, dtype=np.uint8)
        self._call(self.L.ect_set_mesh, _ptr(xyz), xyz.shape[0], _ptr(tets), tets.shape[0], _ptr(sigma),
                   _ptr(nu), _ptr(sd), _ptr(nd), _ptr(bon), _ptr(bc))
        self.n_nodes = xyz.shape[0]

    def set_defect(self, sigma_d, nu_d):
        sd = None if sigma_d is None else np.ascontiguousarray(sigma_d, dtype=np.float64)
        nd = None if nu_d is None else np.ascontiguousarray(nu_d, dtype=np.float64)
        self._call(self.L.ect_set_defect, _ptr(sd), _ptr(nd))

    def set_ibc(self, which, plate, sigma_p, nu_p):
        """Impedance boundary condition on the surface of the tets flagged in `plate` (None clears)."""
        arr = None if plate is None else np.ascontiguousarray(plate, dtype=np.uint8)
        self._call(self.L.ect_set_ibc, int(which), None if arr is None else _ptr(arr), float(sigma_p), float(nu_p))

    def set_physics(self, freq_hz, nu_tilde, delta_gauge):
        self._call(self.L.ect_set_physics, float(freq_hz), float(nu_tilde), float(delta_gauge))

    def load_problem(self, p):
        """set_mesh + set_physics from an object with the fields of a problem description."""
        m = p.mesh
        self.set_mesh(m.xyz, m.tets, p.sigma, p.nu, p.sigma_d, p.nu_d, m.block_of_node, m.bc_mask)
        self.set_physics(p.freq, p.nu_tilde, p.delta)

    # ---- assembly and preconditioner ---------------------------------------
    def assemble(self, which, precision_mask=ECT_F64):
        self._call(self.L.ect_assemble, int(which), int(precision_mask))

    def precond_setup(self, which, precision_mask=ECT_F64, coarse_group=-1):
        self._call(self.L.ect_precond_setup, int(which), int(precision_mask), int(coarse_group))

    def matrix_info(self):
        n, nb = ctypes.c_int64(), ctypes.c_int64()
        rc = self.L.ect_matrix_info(self.h, ctypes.byref(n), ctypes.byref(nb))
        if rc != ECT_OK:
            raise EctError(rc, "matrix_info")
        return n.value, nb.value

    def matrix_copy(self, which):
        n, nb = self.matrix_info()
        rp = np.empty(n + 1, dtype=np.int32)
        col = np.empty(nb, dtype=np.int32)
        val = np.empty((nb, 4, 4, 2), dtype=np.float64)
        self._call(self.L.ect_matrix_copy, int(which), _ptr(rp), _ptr(col), _ptr(val))
        return rp, col, val[..., 0] + 1j * val[..., 1]

    def scaling_copy(self, which):
        t = np.empty(4 * self.n_nodes, dtype=np.float64)
        self._call(self.L.ect_scaling_copy, int(which), _ptr(t))
        return t

    # ---- kernels -------------------------------------------------------------
    def spmv(self, which, x, y, k=1, precision=ECT_F64):
        self._call(self.L.ect_spmv, int(which), int(precision), _dptr(x), _dptr(y), int(k))

    def set_block_split(self, parts):
        self._call(self.L.ect_set_block_split, int(parts))

    def block_split(self):
        return int(self.L.ect_get_block_split(self.h))

    def set_spmm_rows(self, rows):
        self._call(self.L.ect_set_spmm_rows, int(rows))

    def precond_apply(self, which, r, z, k=1, precision=ECT_F64):
        self._call(self.L.ect_precond_apply, int(which), int(precision), _dptr(r), _dptr(z), int(k))

    def cgs2(self, V, w, precision=ECT_F64):
        """V: (j, n) tensor of orthonormal rows, w: (n,) tensor (overwritten)."""
        j, n = V.shape
        h = np.empty((j, 2), dtype=np.float64)
        beta = np.empty(1, dtype=np.float64)
        self._call(self.L.ect_cgs2, int(precision), _dptr(V), int(j), int(n), _dptr(w), _ptr(h), _ptr(beta))
        return h[:, 0] + 1j * h[:, 1], float(beta[0])

    def coil_rhs(self, c, z_probe, out):
        z = np.ascontiguousarray(np.atleast_1d(z_probe), dtype=np.float64)
        cc = coil(c)
        self._call(self.L.ect_coil_rhs, ctypes.byref(cc), _ptr(z), int(z.size), _dptr(out))

    def solve(self, which, rhs, x, k=1, options=None):
        o = options if options is not None else default_options()
        st = Stats()
        try:
            self._call(self.L.ect_solve, int(which), _dptr(rhs), _dptr(x), int(k), ctypes.byref(o),
                       ctypes.byref(st), stats=st)
        except EctError as e:
            e.stats = st.as_dict()
            raise
        return st.as_dict()

    def autotune(self, which, rhs, work, k, base=None):
        """Pick rhs_tile, restart and inner_iters for this workload; returns (options, stats)."""
        o = base if base is not None else default_options()
        best = Options()
        st = Stats()
        self._call(self.L.ect_autotune, int(which), _dptr(rhs), _dptr(work), int(k), ctypes.byref(o),
                   ctypes.byref(best), ctypes.byref(st))
        return best, st.as_dict()

    def delta_z(self, u0, ud, b, currents):
        cur = np.ascontiguousarray(currents, dtype=np.float64)
        dz = np.empty((2, 2, 2), dtype=np.float64)
        dze = np.empty((2, 2, 2), dtype=np.float64)
        self._call(self.L.ect_delta_z, _dptr(u0), _dptr(ud), None if b is None else _dptr(b), _ptr(cur),
                   _ptr(dz), _ptr(dze) if b is not None else None)
        out = dz[..., 0] + 1j * dz[..., 1]
        return out, (dze[..., 0] + 1j * dze[..., 1]) if b is not None else None

    def delta_z_static(self, u0, ud, b, currents, n_pos):
        """Delta Z for n_pos positions ([n_pos][2][4N] tensors) with no device allocation."""
        cur = np.ascontiguousarray(currents, dtype=np.float64)
        dz = np.empty((n_pos, 2, 2, 2), dtype=np.float64)
        dze = np.empty((n_pos, 2, 2, 2), dtype=np.float64)
        self._call(self.L.ect_delta_z_static, _dptr(u0), _dptr(ud), None if b is None else _dptr(b), _ptr(cur),
                   int(n_pos), _ptr(dz), _ptr(dze) if b is not None else None)
        out = dz[..., 0] + 1j * dz[..., 1]
        return out, (dze[..., 0] + 1j * dze[..., 1]) if b is not None else None

    def impedance(self, coils, z_pos, options=None):
        z = np.ascontiguousarray(np.atleast_1d(z_pos), dtype=np.float64)
        arr = (Coil * 2)(coil(coils[0]), coil(coils[1]))
        o = options if options is not None else default_options()
        dz = np.empty((z.size, 2, 2, 2), dtype=np.float64)
        st = Stats()
        try:
            self._call(self.L.ect_impedance, arr, _ptr(z), int(z.size), ctypes.byref(o), _ptr(dz),
                       ctypes.byref(st), stats=st)
        except EctError as e:
            e.stats = st.as_dict()
            raise
        return dz[..., 0] + 1j * dz[..., 1], st.as_dict()


    def assemble_sweep(self, freqs_hz, precision_mask=ECT_F64):
        f = np.ascontiguousarray(np.atleast_1d(freqs_hz), dtype=np.float64)
        self._call(self.L.ect_assemble_sweep, _ptr(f), int(f.size), int(precision_mask))
        self.n_sweep = int(f.size)

    def solve_sweep(self, config, rhs, x, k, options=None):
        o = options if options is not None else default_options()
        st = Stats()
        try:
            self._call(self.L.ect_solve_sweep, int(config), _dptr(rhs), _dptr(x), int(k), ctypes.byref(o),
                       ctypes.byref(st), stats=st)
        except EctError as e:
            e.stats = st.as_dict()
            raise
        return st.as_dict()

    def impedance_sweep(self, coils, z_pos, options=None):
        z = np.ascontiguousarray(np.atleast_1d(z_pos), dtype=np.float64)
        arr = (Coil * 2)(coil(coils[0]), coil(coils[1]))
        o = options if options is not None else default_options()
        dz = np.empty((self.n_sweep, z.size, 2, 2, 2), dtype=np.float64)
        st = Stats()
        self._call(self.L.ect_impedance_sweep, arr, _ptr(z), int(z.size), ctypes.byref(o), _ptr(dz),
                   ctypes.byref(st), stats=st)
        return dz[..., 0] + 1j * dz[..., 1], st.as_dict()


MLP_SIZES = (6, 256, 256, 256, 256, 256)


def mlp_flatten(layers):
    """[(W (out x in), b (out)), ...] -> flat float32 parameter vector (W row-major, then b, per layer)."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32)])
                           for W, b in layers]).astype(np.float32)


def mlp_unflatten(v, sizes=MLP_SIZES):
    out, o = [], 0
    for i in range(len(sizes) - 1):
        fi, fo = sizes[i], sizes[i + 1]
        W = v[o:o + fi * fo].reshape(fo, fi)
        o += fi * fo
        b = v[o:o + fo]
        o += fo
        out.append((W, b))
    return out


class Surrogate:
    """The tcgen05 surrogate MLP (ect_mlp_*) on its own CUDA stream."""

    def __init__(self, batch=256):
        import torch
        self._torch = torch
        self.L = load_library()
        self.stream = torch.cuda.Stream()
        h = ctypes.c_void_p()
        rc = self.L.ect_mlp_create(ctypes.byref(h), ctypes.c_void_p(self.stream.cuda_stream), int(batch))
        if rc != ECT_OK:
            raise EctError(rc, self.L.ect_mlp_last_error(None).decode())
        self.h = h
        self.batch = batch
        self.n_params = self.L.ect_mlp_num_params()

    def close(self):
        if getattr(self, "h", None):
            self.L.ect_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, fn, *args):
        cur = self._torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        rc = fn(self.h, *args)
        cur.wait_stream(self.stream)
        if rc != ECT_OK:
            raise EctError(rc, self.L.ect_mlp_last_error(self.h).decode())

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.n_params
        self._call(self.L.ect_mlp_set_params, _ptr(flat))

    def get_params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        self._call(self.L.ect_mlp_get_params, _ptr(out))
        return out

    def forward(self, x, y):
        self._call(self.L.ect_mlp_forward, _dptr(x), _dptr(y))

    def gradients(self, x, t):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = np.empty(1, dtype=np.float64)
        self._call(self.L.ect_mlp_gradients, _dptr(x), _dptr(t), _ptr(g), _ptr(loss))
        return g, float(loss[0])

    def train_step(self, x, t, lr, want_loss=False):
        loss = np.empty(1, dtype=np.float64)
        self._call(self.L.ect_mlp_train_step, _dptr(x), _dptr(t), ctypes.c_float(lr),
                   _ptr(loss) if want_loss else None)
        return float(loss[0]) if want_loss else None
