"""Python binding of libsplitsolve.so (argument marshalling only).

Every computation happens in the CUDA library behind ``include/splitsolve.h``;
this module converts numpy arrays / torch tensors to pointers and back.  If
the shared library has not been built, importing still works but every call
raises ``RuntimeError`` -- there is no CPU fallback.

Names follow the C ABI: :func:`ss_create`, :meth:`Handle.set_hamiltonian`
(``ss_set_hamiltonian``), :meth:`Handle.self_energy` (``ss_self_energy``),
:meth:`Handle.solve` (``ss_solve``), :meth:`Handle.transmission`
(``ss_transmission``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsplitsolve.so")

SS_OK, SS_ERR_ARG, SS_ERR_STATE, SS_ERR_SINGULAR, SS_ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
SS_ERR_TIMEOUT, SS_ERR_OOM, SS_ERR_CUDA = 5, 6, 7
SS_FP64, SS_MIXED_BF16X3, SS_MIXED_BF16X6, SS_MIXED_OZAKI = 0, 1, 2, 3
SS_OBC_DECIMATION, SS_OBC_FEAST = 0, 1
STATUS_NAMES = {0: "SS_OK", 1: "SS_ERR_ARG", 2: "SS_ERR_STATE", 3: "SS_ERR_SINGULAR",
                4: "SS_ERR_NOT_CONVERGED", 5: "SS_ERR_TIMEOUT", 6: "SS_ERR_OOM", 7: "SS_ERR_CUDA"}

EXPORTS = ("ss_config_default", "ss_create", "ss_set_hamiltonian", "ss_self_energy", "ss_solve",
           "ss_transmission", "ss_destroy", "ss_last_error", "ss_launch_count", "ss_profile_read",
           "ss_profile_reset", "ss_profile_read_issued", "ss_zgemm", "ss_caroli_transmission",
           "ss_caroli_transmission_noalloc", "ss_noalloc_last_error", "ss_mlp_create", "ss_mlp_destroy",
           "ss_mlp_set_params", "ss_mlp_get", "ss_mlp_forward", "ss_mlp_train_step", "ss_mlp_last_error",
           "ss_mlp_use_tensor_cores", "ss_set_warm_start", "ss_surface_gf", "ss_autotune", "ss_exact_gemm_plan", "ss_dos",
           "ss_set_momentum", "ss_host_launch_count")
KERNEL_KINDS = {"zgemm": 0, "form": 1, "lu_panel": 2, "lu_row": 3, "lu_back": 4, "norm1": 5, "trace": 6,
                "check": 7, "fill": 8, "tc_pack_a": 9, "tc_pack_b": 10, "tcgemm": 11, "zgemm32": 12,
                "oz_scale": 13, "oz_pack": 14, "ozgemm": 15, "frob2": 16, "zgemm_lu": 17, "ozgemm_lu": 18,
                "lu_hpanel": 19, "eig": 20}


class SSConfig(C.Structure):
    _fields_ = [
        ("n_b_max", C.c_int), ("s_b_max", C.c_int), ("max_points", C.c_int), ("max_inj", C.c_int),
        ("precision", C.c_int), ("eta", C.c_double), ("decim_tol", C.c_double),
        ("decim_max_iter", C.c_int), ("ir_tol", C.c_double), ("ir_max_iter", C.c_int),
        ("warm_start", C.c_int), ("stream", C.c_void_p), ("device_ptrs", C.c_int),
        ("use_graphs", C.c_int), ("profile", C.c_int), ("partitions", C.c_int), ("memory_lean", C.c_int),
        ("hermitian_sweeps", C.c_int), ("obc", C.c_int), ("feast_radius", C.c_double),
        ("feast_points", C.c_int), ("feast_subspace", C.c_int), ("tournament_pivoting", C.c_int),
        ("lu_lookahead", C.c_int),
    ]


class SSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib_handle = None


def load_library(path: str = LIB_PATH):
    """Load the shared library (raises if it is missing: no CPU fallback)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    lib.ss_config_default.argtypes = [C.POINTER(SSConfig)]
    lib.ss_config_default.restype = None
    lib.ss_create.argtypes = [C.POINTER(vp), C.POINTER(SSConfig)]
    lib.ss_set_hamiltonian.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp]
    lib.ss_self_energy.argtypes = [vp, C.c_int, dp, ip, vp, vp, ip, ip]
    lib.ss_solve.argtypes = [vp, C.c_int, dp, ip, C.c_int, vp, vp, ip]
    lib.ss_transmission.argtypes = [vp, C.c_int, dp, ip, vp, vp, ip]
    lib.ss_dos.argtypes = [vp, C.c_int, dp, ip, vp, ip]
    lib.ss_dos.restype = C.c_int
    lib.ss_destroy.argtypes = [vp]
    lib.ss_last_error.argtypes = [vp]
    lib.ss_last_error.restype = C.c_char_p
    lib.ss_launch_count.argtypes = [vp]
    lib.ss_launch_count.restype = C.c_longlong
    lib.ss_host_launch_count.argtypes = [vp]
    lib.ss_host_launch_count.restype = C.c_longlong
    lib.ss_profile_read.argtypes = [vp, C.c_int, dp, dp, C.POINTER(C.c_longlong)]
    lib.ss_profile_read.restype = C.c_int
    lib.ss_profile_read_issued.argtypes = [vp, C.c_int, dp]
    lib.ss_profile_read_issued.restype = C.c_int
    lib.ss_profile_reset.argtypes = [vp]
    lib.ss_profile_reset.restype = C.c_int
    lib.ss_zgemm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, C.c_int, vp, C.c_int, C.c_int, vp,
                             C.c_int, vp]
    lib.ss_zgemm.restype = C.c_int
    lib.ss_caroli_transmission.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp]
    lib.ss_caroli_transmission.restype = C.c_int
    lib.ss_caroli_transmission_noalloc.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp]
    lib.ss_caroli_transmission_noalloc.restype = C.c_int
    lib.ss_noalloc_last_error.argtypes = []
    lib.ss_noalloc_last_error.restype = C.c_char_p
    fp = C.POINTER(C.c_float)
    lib.ss_mlp_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_int, C.c_ulonglong, vp]
    lib.ss_mlp_destroy.argtypes = [vp]
    lib.ss_mlp_set_params.argtypes = [vp, C.POINTER(vp), C.c_int]
    lib.ss_mlp_get.argtypes = [vp, C.c_int, C.POINTER(vp)]
    lib.ss_mlp_forward.argtypes = [vp, C.c_int, vp, vp]
    lib.ss_mlp_train_step.argtypes = [vp, C.c_int, vp, vp, C.c_float, dp]
    lib.ss_mlp_use_tensor_cores.argtypes = [vp, C.c_int]
    lib.ss_mlp_last_error.argtypes = [vp]
    lib.ss_mlp_last_error.restype = C.c_char_p
    lib.ss_set_warm_start.argtypes = [vp, vp, C.c_int, C.c_double]
    lib.ss_set_momentum.argtypes = [vp, C.c_int, C.c_double]
    lib.ss_set_momentum.restype = C.c_int
    lib.ss_autotune.argtypes = [vp, C.c_int, C.c_int, C.c_char_p, ip, ip, ip, dp]
    lib.ss_autotune.restype = C.c_int
    ub = C.POINTER(C.c_ubyte)
    lib.ss_exact_gemm_plan.argtypes = [C.c_int, ip, ip, ip, ip, ub, ub, ub]
    lib.ss_exact_gemm_plan.restype = C.c_int
    lib.ss_surface_gf.argtypes = [vp, C.c_int, dp, ip, dp, C.c_int, C.c_int, C.c_int, C.c_double, vp, ip, ip, ip]
    for name in ("ss_mlp_create", "ss_mlp_destroy", "ss_mlp_set_params", "ss_mlp_get", "ss_mlp_forward",
                 "ss_mlp_train_step", "ss_mlp_use_tensor_cores", "ss_set_warm_start", "ss_surface_gf"):
        getattr(lib, name).restype = C.c_int
    for name in ("ss_create", "ss_set_hamiltonian", "ss_self_energy", "ss_solve", "ss_transmission",
                 "ss_destroy"):
        getattr(lib, name).restype = C.c_int
    _lib_handle = lib
    return lib


def ss_config_default() -> SSConfig:
    cfg = SSConfig()
    load_library().ss_config_default(C.byref(cfg))
    return cfg


def _ptr(a):
    """Pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _host_c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dev_in(t):
    """Device input: the library reads dense row-major blocks, so make it contiguous."""
    return t if t.is_contiguous() else t.contiguous()


def _dev_out(t):
    if not t.is_contiguous():
        raise ValueError("output tensors must be contiguous (dense row-major)")
    return t


class Handle:
    """Owns one ``ss_handle``.  With ``device_ptrs=True`` array arguments are
    torch CUDA tensors (complex128 / float64); otherwise numpy arrays."""

    def __init__(self, **kw):
        lib = load_library()
        cfg = ss_config_default()
        for k, v in kw.items():
            if not hasattr(cfg, k):
                raise TypeError(f"unknown config field {k}")
            setattr(cfg, k, v)
        self.cfg = cfg
        self.device_ptrs = bool(cfg.device_ptrs)
        h = C.c_void_p()
        rc = lib.ss_create(C.byref(h), C.byref(cfg))
        if rc != SS_OK:
            raise SSError(rc, lib.ss_last_error(None).decode())
        self._h = h
        self._lib = lib
        self.shapes = {}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ss_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self._lib.ss_last_error(self._h).decode()

    def launch_count(self) -> int:
        return int(self._lib.ss_launch_count(self._h))

    def host_launch_count(self) -> int:
        """ss_host_launch_count: host-side launch calls (eager kernels, memsets, graph launches)."""
        return int(self._lib.ss_host_launch_count(self._h))

    def profile_read(self, kind):
        """(total_ms, flops, launches) of one kernel kind (needs profile=1)."""
        ms, fl, n = C.c_double(), C.c_double(), C.c_longlong()
        k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
        self._check(self._lib.ss_profile_read(self._h, k, C.byref(ms), C.byref(fl), C.byref(n)))
        return ms.value, fl.value, n.value

    def profile_issued(self, kind):
        """Tensor-pipe flops issued by a kernel kind (needs profile=1)."""
        v = C.c_double()
        k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
        self._check(self._lib.ss_profile_read_issued(self._h, k, C.byref(v)))
        return v.value

    def profile_reset(self):
        self._check(self._lib.ss_profile_reset(self._h))

    def _check(self, rc, allow=()):
        if rc != SS_OK and rc not in allow:
            raise SSError(rc, self.last_error())
        return rc

    # ------------------------------------------------------------------ calls
    def set_hamiltonian(self, k_id, H_diag, H_up, S_diag, S_up, lead_L=None, lead_R=None):
        """ss_set_hamiltonian; arrays (n_b,s,s), (n_b-1,s,s); leads (4,s,s) or None."""
        n_b, s = int(H_diag.shape[0]), int(H_diag.shape[1])
        if not self.device_ptrs:
            H_diag, S_diag = _host_c128(H_diag), _host_c128(S_diag)
            H_up, S_up = _host_c128(H_up), _host_c128(S_up)
            lead_L = None if lead_L is None else _host_c128(lead_L)
            lead_R = None if lead_R is None else _host_c128(lead_R)
        else:
            H_diag, S_diag, H_up, S_up = _dev_in(H_diag), _dev_in(S_diag), _dev_in(H_up), _dev_in(S_up)
            lead_L = None if lead_L is None else _dev_in(lead_L)
            lead_R = None if lead_R is None else _dev_in(lead_R)
        rc = self._lib.ss_set_hamiltonian(self._h, int(k_id), n_b, s, _ptr(H_diag), _ptr(H_up), _ptr(S_diag),
                                          _ptr(S_up), _ptr(lead_L), _ptr(lead_R))
        self._check(rc)
        self.shapes[int(k_id)] = (n_b, s)

    def set_device(self, k_id, dev):
        """set_hamiltonian from a ``synth.Device`` (numpy, host mode only)."""
        lead = lambda t: None if t is None else np.stack(t)
        self.set_hamiltonian(k_id, dev.H_diag, dev.H_up, dev.S_diag, dev.S_up, lead(dev.lead_L),
                             lead(dev.lead_R))

    def _pts(self, E, k_id):
        E = np.ascontiguousarray(np.atleast_1d(E), dtype=np.float64)
        k = np.ascontiguousarray(np.broadcast_to(np.atleast_1d(k_id), E.shape), dtype=np.int32)
        return E, k

    def _alloc(self, count, dtype):
        if self.device_ptrs:
            import torch
            tdt = torch.complex128 if dtype == np.complex128 else torch.float64
            return torch.zeros(count, dtype=tdt, device="cuda")
        return np.zeros(count, dtype)

    def self_energy(self, E, k_id, allow=(SS_ERR_NOT_CONVERGED, SS_ERR_SINGULAR)):
        """Returns (Sigma_L, Sigma_R, iters (P,2), status (P,), rc)."""
        E, k = self._pts(E, k_id)
        P = E.size
        sizes = [self.shapes[int(q)][1] ** 2 for q in k]
        tot = int(sum(sizes))
        sL = self._alloc(tot, np.complex128)
        sR = self._alloc(tot, np.complex128)
        it = np.zeros(2 * P, np.int32)
        st = np.zeros(P, np.int32)
        rc = self._lib.ss_self_energy(self._h, P, E.ctypes.data_as(C.POINTER(C.c_double)),
                                      k.ctypes.data_as(C.POINTER(C.c_int)), _ptr(sL), _ptr(sR),
                                      it.ctypes.data_as(C.POINTER(C.c_int)), st.ctypes.data_as(C.POINTER(C.c_int)))
        self._check(rc, allow)
        return self._split(sL, k), self._split(sR, k), it.reshape(P, 2), st, rc

    def _split(self, flat, k):
        out, o = [], 0
        for q in k:
            s = self.shapes[int(q)][1]
            out.append(flat[o:o + s * s].reshape(s, s))
            o += s * s
        return out

    def solve(self, E, k_id, inj, allow=(SS_ERR_NOT_CONVERGED, SS_ERR_SINGULAR), want_x=True):
        """ss_solve; inj: list of (2s, n_inj) per point (or one packed array).

        Returns (x list of (n_b*s, n_inj), status, rc)."""
        E, k = self._pts(E, k_id)
        P = E.size
        if isinstance(inj, (list, tuple)):
            n_inj = int(inj[0].shape[1])
            if self.device_ptrs:
                import torch
                flat = torch.cat([t.reshape(-1) for t in inj])
            else:
                flat = np.concatenate([_host_c128(a).reshape(-1) for a in inj])
        else:
            n_inj = int(inj.shape[-1])
            flat = inj.reshape(-1) if self.device_ptrs else _host_c128(inj).reshape(-1)
        xs = sum(self.shapes[int(q)][0] * self.shapes[int(q)][1] for q in k) * n_inj
        x = self._alloc(xs, np.complex128) if want_x else None
        st = np.zeros(P, np.int32)
        rc = self._lib.ss_solve(self._h, P, E.ctypes.data_as(C.POINTER(C.c_double)),
                                k.ctypes.data_as(C.POINTER(C.c_int)), n_inj, _ptr(flat), _ptr(x),
                                st.ctypes.data_as(C.POINTER(C.c_int)))
        self._check(rc, allow)
        out = None
        if want_x:
            out, o = [], 0
            for q in k:
                n, s = self.shapes[int(q)]
                out.append(x[o:o + n * s * n_inj].reshape(n * s, n_inj))
                o += n * s * n_inj
        return out, st, rc

    def autotune(self, s_b, n_problems, cache_path=None):
        """ss_autotune: returns (panel width, outer width (0: one level), update arithmetic, ms)."""
        nb, nbo, upd, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        cp = None if cache_path is None else str(cache_path).encode()
        self._check(self._lib.ss_autotune(self._h, int(s_b), int(n_problems), cp, C.byref(nb), C.byref(nbo),
                                          C.byref(upd), C.byref(ms)))
        return nb.value, nbo.value, upd.value, ms.value

    def set_momentum(self, k_id, k):
        """ss_set_momentum: transverse momentum of k_id fed to the warm-start network."""
        self._check(self._lib.ss_set_momentum(self._h, int(k_id), float(k)))

    def set_warm_start(self, net, side, out_scale):
        """ss_set_warm_start: attach a trained MLP to lead `side` (0 left, 1 right)."""
        self._check(self._lib.ss_set_warm_start(self._h, net._n, int(side), float(out_scale)))
        self._warm = net  # keep it alive while attached

    def surface_gf(self, E, k_id, kval=None, side=1, use_warm=False, warm_iters=8, warm_tol=1e-10,
                   allow=(SS_ERR_NOT_CONVERGED, SS_ERR_SINGULAR)):
        """ss_surface_gf; returns (g list of (s,s), iters, seeded, status, rc)."""
        E, k = self._pts(E, k_id)
        P = E.size
        kv = None if kval is None else np.ascontiguousarray(np.broadcast_to(np.atleast_1d(kval), E.shape),
                                                            dtype=np.float64)
        tot = int(sum(self.shapes[int(q)][1] ** 2 for q in k))
        g = self._alloc(tot, np.complex128)
        it = np.zeros(P, np.int32)
        sd = np.zeros(P, np.int32)
        st = np.zeros(P, np.int32)
        rc = self._lib.ss_surface_gf(self._h, P, E.ctypes.data_as(C.POINTER(C.c_double)),
                                     k.ctypes.data_as(C.POINTER(C.c_int)),
                                     None if kv is None else kv.ctypes.data_as(C.POINTER(C.c_double)), int(side),
                                     int(bool(use_warm)), int(warm_iters), float(warm_tol), _ptr(g),
                                     it.ctypes.data_as(C.POINTER(C.c_int)), sd.ctypes.data_as(C.POINTER(C.c_int)),
                                     st.ctypes.data_as(C.POINTER(C.c_int)))
        self._check(rc, allow)
        return self._split(g, k), it, sd, st, rc

    def dos(self, E, k_id, allow=(SS_ERR_NOT_CONVERGED, SS_ERR_SINGULAR)):
        """ss_dos: local density of states -Im Tr[G_ii]/pi per block.

        Returns (list of (n_b,) arrays, status (P,), rc)."""
        E, k = self._pts(E, k_id)
        P = E.size
        tot = int(sum(self.shapes[int(q)][0] for q in k))
        out = self._alloc(tot, np.float64)
        st = np.zeros(P, np.int32)
        rc = self._lib.ss_dos(self._h, P, E.ctypes.data_as(C.POINTER(C.c_double)),
                              k.ctypes.data_as(C.POINTER(C.c_int)), _ptr(out), st.ctypes.data_as(C.POINTER(C.c_int)))
        self._check(rc, allow)
        res, o = [], 0
        for q in k:
            n = self.shapes[int(q)][0]
            res.append(out[o:o + n])
            o += n
        return res, st, rc

    def transmission(self, E, k_id, allow=(SS_ERR_NOT_CONVERGED, SS_ERR_SINGULAR)):
        """Returns (T (P,), err_est (P,), status (P,), rc)."""
        E, k = self._pts(E, k_id)
        P = E.size
        T = self._alloc(P, np.float64)
        err = self._alloc(P, np.float64)
        st = np.zeros(P, np.int32)
        rc = self._lib.ss_transmission(self._h, P, E.ctypes.data_as(C.POINTER(C.c_double)),
                                       k.ctypes.data_as(C.POINTER(C.c_int)), _ptr(T), _ptr(err),
                                       st.ctypes.data_as(C.POINTER(C.c_int)))
        self._check(rc, allow)
        return T, err, st, rc


def ss_create(**kw) -> Handle:
    return Handle(**kw)


def ss_zgemm(A, B, C, precision=SS_FP64, transA=False, transB=False, stream=None):
    """C = op(A) op(B) with the library kernels (torch CUDA complex128 tensors, row-major)."""
    lib = load_library()
    A, B, C = _dev_in(A), _dev_in(B), _dev_out(C)
    m = int(A.shape[1] if transA else A.shape[0])
    k = int(A.shape[0] if transA else A.shape[1])
    n = int(B.shape[0] if transB else B.shape[1])
    rc = lib.ss_zgemm(int(precision), m, n, k, _ptr(A), int(A.stride(0)), int(transA), _ptr(B), int(B.stride(0)),
                      int(transB), _ptr(C), int(C.stride(0)), stream)
    if rc != SS_OK:
        raise SSError(rc, lib.ss_last_error(None).decode())


def exact_gemm_plan(k):
    """ss_exact_gemm_plan: (w, beta, S, passes) with passes a list of
    (level, first t, number of pairs) for inner dimension k (no GPU needed)."""
    lib = load_library()
    w, beta, S, npass = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    pd, pt0, pnp = (C.c_ubyte * 64)(), (C.c_ubyte * 64)(), (C.c_ubyte * 64)()
    rc = lib.ss_exact_gemm_plan(int(k), C.byref(w), C.byref(beta), C.byref(S), C.byref(npass), pd, pt0, pnp)
    if rc != SS_OK:
        raise SSError(rc, "no exact split for k = %d" % k)
    return w.value, beta.value, S.value, [(pd[p], pt0[p], pnp[p]) for p in range(npass.value)]


def _check_caroli_args(sigma_L, sigma_R, G1n, T):
    """Host-side checks of the Caroli entry points' tensors, so that nothing the
    kernels would read or write out of bounds reaches the device: CUDA tensors
    on the current device, complex128 blocks of one shape (P, s, s), a float64
    T of at least P entries.  Returns (P, s)."""
    import torch
    named = (("sigma_L", sigma_L), ("sigma_R", sigma_R), ("G1n", G1n), ("T", T))
    for name, t in named:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
    cur = torch.cuda.current_device()
    for name, t in named:
        if t.device.index != cur:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
    for name, t in named[:3]:
        if t.dtype != torch.complex128:
            raise ValueError(f"{name} must be complex128, got {t.dtype}")
    if T.dtype != torch.float64:
        raise ValueError(f"T must be float64, got {T.dtype}")
    if sigma_L.dim() != 3 or sigma_L.shape[1] != sigma_L.shape[2] or sigma_L.shape[1] < 1:
        raise ValueError(f"sigma_L must have shape (P, s, s), got {tuple(sigma_L.shape)}")
    for name, t in named[1:3]:
        if tuple(t.shape) != tuple(sigma_L.shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, sigma_L has {tuple(sigma_L.shape)}")
    P, s = int(sigma_L.shape[0]), int(sigma_L.shape[1])
    if T.numel() < P:
        raise ValueError(f"T holds {T.numel()} entries, {P} are written")
    return P, s


def ss_caroli_transmission(sigma_L, sigma_R, G1n, T, stream=None):
    """T[p] = Re Tr[Gamma_L G Gamma_R G^H]; torch CUDA tensors (P,s,s) complex128 and (P,) float64."""
    lib = load_library()
    _check_caroli_args(sigma_L, sigma_R, G1n, T)
    sigma_L, sigma_R, G1n, T = _dev_in(sigma_L), _dev_in(sigma_R), _dev_in(G1n), _dev_out(T)
    P, s = int(sigma_L.shape[0]), int(sigma_L.shape[1])
    rc = lib.ss_caroli_transmission(P, s, _ptr(sigma_L), _ptr(sigma_R), _ptr(G1n), _ptr(T), stream)
    if rc != SS_OK:
        raise SSError(rc, lib.ss_last_error(None).decode())


def ss_caroli_transmission_noalloc(sigma_L, sigma_R, G1n, T, stream=None):
    """Allocation-free Caroli transmission (scratch in a fixed device array).

    For callers that cannot allocate device memory; same result as
    :func:`ss_caroli_transmission`.  Limits: P <= 256, P*s^2 <= 65536.
    Inputs must already be contiguous: copying them would allocate."""
    lib = load_library()
    P, s = _check_caroli_args(sigma_L, sigma_R, G1n, T)
    for t in (sigma_L, sigma_R, G1n, T):
        if not t.is_contiguous():
            raise ValueError("inputs and outputs must be contiguous (dense row-major)")
    rc = lib.ss_caroli_transmission_noalloc(P, s, _ptr(sigma_L), _ptr(sigma_R), _ptr(G1n), _ptr(T), stream)
    if rc != SS_OK:
        raise SSError(rc, lib.ss_noalloc_last_error().decode())


class MLP:
    """Warm-start network run by the library's kernels (ss_mlp_*).

    Arrays passed to forward/train_step are torch CUDA float32 tensors."""

    def __init__(self, n_in, width, n_out, max_batch, seed=0, stream=None):
        lib = load_library()
        n = C.c_void_p()
        rc = lib.ss_mlp_create(C.byref(n), int(n_in), int(width), int(n_out), int(max_batch), int(seed), stream)
        if rc != SS_OK:
            raise SSError(rc, "ss_mlp_create failed")
        self._n, self._lib = n, lib
        self.n_in, self.width, self.n_out, self.max_batch = n_in, width, n_out, max_batch
        self.shapes = [(width, n_in), (width,), (width, width), (width,), (n_out, width), (n_out,)]

    def close(self):
        if getattr(self, "_n", None):
            self._lib.ss_mlp_destroy(self._n)
            self._n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != SS_OK:
            raise SSError(rc, self._lib.ss_mlp_last_error(self._n).decode())

    def set_params(self, params):
        arrs = [np.ascontiguousarray(p, dtype=np.float32) for p in params]
        ptrs = (C.c_void_p * 6)(*[a.ctypes.data for a in arrs])
        self._check(self._lib.ss_mlp_set_params(self._n, ptrs, 0))

    def _get(self, which):
        out = [np.zeros(sh, np.float32) for sh in self.shapes]
        ptrs = (C.c_void_p * 6)(*[a.ctypes.data for a in out])
        self._check(self._lib.ss_mlp_get(self._n, which, ptrs))
        return out

    def get_params(self):
        return self._get(0)

    def use_tensor_cores(self, on):
        """GEMMs on the tcgen05 tensor cores (default when width and n_out are
        multiples of 8) or on the SIMT kernel."""
        self._check(self._lib.ss_mlp_use_tensor_cores(self._n, int(bool(on))))

    def get_grads(self):
        return self._get(1)

    def forward(self, x):
        import torch
        x = _dev_in(x)
        y = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=x.device)
        self._check(self._lib.ss_mlp_forward(self._n, int(x.shape[0]), _ptr(x), _ptr(y)))
        return y

    def train_step(self, x, t, lr):
        x, t = _dev_in(x), _dev_in(t)
        loss = C.c_double()
        self._check(self._lib.ss_mlp_train_step(self._n, int(x.shape[0]), _ptr(x), _ptr(t), float(lr),
                                                C.byref(loss)))
        return loss.value
