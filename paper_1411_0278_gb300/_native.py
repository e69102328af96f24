"""Thin ctypes binding of libgbi (include/gbi.h): argument marshalling only.

Every computation happens inside libgbi's CUDA kernels.  Device arrays are torch
float64 CUDA tensors whose ``data_ptr()`` is passed through; outputs are
allocated with torch.  If the shared library has not been built, the first call
raises ``ImportError`` -- there is no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgbi.so")

GBI_OK, GBI_ERR_ARG, GBI_ERR_OVERLAP, GBI_ERR_NOT_CONVERGED, GBI_ERR_TIMEOUT, GBI_ERR_CUDA, GBI_ERR_NOMEM = range(7)
SET_ALL, SET_L, SET_H = 0, 1, 2

c_double_p = ctypes.POINTER(ctypes.c_double)


class gbi_params(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("eta", ctypes.c_double), ("trunc", ctypes.c_int),
                ("precision", ctypes.c_int), ("rtol", ctypes.c_double), ("restart", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("max_refine", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("min_sep", ctypes.c_double)]


class gbi_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refinements", ctypes.c_int), ("matvecs_f32", ctypes.c_int),
                ("matvecs_f64", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("min_separation", ctypes.c_double), ("pair_interactions", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GbiError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__("%s: %s (%d)%s" % (where, status_string(status), status,
                                           (": " + detail) if detail else ""))


_LIB = None
_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGS = {
    "gbi_create": (_I, [ctypes.POINTER(_VP), _I]),
    "gbi_destroy": (_I, [_VP]),
    "gbi_set_stream": (_I, [_VP, _VP]),
    "gbi_synchronize": (_I, [_VP]),
    "gbi_status_string": (ctypes.c_char_p, [_I]),
    "gbi_last_error": (ctypes.c_char_p, [_VP]),
    "gbi_h": (_I, [_I]),
    "gbi_d": (_I, [_I]),
    "gbi_component_scales": (_I, [_I, c_double_p]),
    "gbi_self_scalars": (_I, [_I, c_double_p]),
    "gbi_apply": (_I, [_VP, _I, _I, _D, _I, _I, _I, _VP, _VP, _VP, _D, _D, _I]),
    "gbi_solve": (_I, [_VP, ctypes.POINTER(gbi_params), _I] + [_VP] * 9 + [_I, ctypes.POINTER(gbi_info)]),
    "gbi_solve_host": (_I, [_VP, ctypes.POINTER(gbi_params), _I] + [_VP] * 9 + [_I, ctypes.POINTER(gbi_info)]),
    "gbi_superpose": (_I, [_VP, ctypes.POINTER(gbi_params), _I] + [_VP] * 8),
    "gbi_trap_inputs": (_I, [_VP, _I, _I, _D, _D, _D, _D] + [_VP] * 7),
    "gbi_trap_step": (_I, [_VP, ctypes.POINTER(gbi_params), _I, _D, _D, _D, _D, _D, _I, _I, _VP, _VP,
                           ctypes.POINTER(gbi_info)]),
    "gbi_squirmer_inputs": (_I, [_VP, _I, _I, _D, _D, _D] + [_VP] * 7),
    "gbi_squirmer_step": (_I, [_VP, ctypes.POINTER(gbi_params), _I, _D, _D, _D, _D, _I, _I, _VP, _VP,
                               ctypes.POINTER(gbi_info)]),
    "gbi_flow": (_I, [_VP, ctypes.POINTER(gbi_params), _I, _VP, _VP, _VP, _VP, _I, _VP, _VP,
                      ctypes.POINTER(ctypes.c_int)]),
    "gbi_batch_trap_step": (_I, [_VP, ctypes.POINTER(gbi_params), _I, ctypes.POINTER(ctypes.c_int), _D, _D, _D, _D,
                                 _D, _I, _I, _VP, _VP, ctypes.POINTER(gbi_info)]),
    "gbi_batch_solve": (_I, [_VP, ctypes.POINTER(gbi_params), _I, ctypes.POINTER(ctypes.c_int)] + [_VP] * 9 +
                        [_I, ctypes.POINTER(gbi_info)]),
    "gbi_batch_superpose": (_I, [_VP, ctypes.POINTER(gbi_params), _I, ctypes.POINTER(ctypes.c_int)] + [_VP] * 8),
    "gbi_solve_static": (_I, [_VP, ctypes.POINTER(gbi_params), _I] + [_VP] * 9 + [_I, ctypes.POINTER(gbi_info)]),
    "gbi_tune": (_I, [_VP, _I, _I, ctypes.POINTER(ctypes.c_int), _I, ctypes.POINTER(ctypes.c_int)]),
    "gbi_set_wpt": (_I, [_VP, _I]),
    "gbi_set_split_tail": (_I, [_VP, _I]),
    "gbi_pass_wpt": (_I, [_VP, _I, _I, _I, _I, _I, _I]),
    "gbi_set_wait_limit": (_I, [_VP, ctypes.c_longlong]),
    "gbi_pass_status": (_I, [_VP]),
    "gbi_pairs": (_I, [_VP, _I, _VP, _D, _D, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "gbi_pairs_get": (_I, [_VP, _VP, _VP]),
    "gbi_mlp_set": (_I, [_VP, _VP, _D]),
    "gbi_mlp_get": (_I, [_VP, _VP, c_double_p]),
    "gbi_mlp_features": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _D, _VP, _VP]),
    "gbi_mlp_forward": (_I, [_VP, _I, _VP, _VP, _VP]),
    "gbi_mlp_set_engine": (_I, [_VP, _I]),
    "gbi_mlp_status": (_I, [_VP]),
    "gbi_mlp_correct": (_I, [_VP, _I, _VP, _VP, _D, _D, _I, ctypes.POINTER(ctypes.c_int), _VP, _VP,
                             ctypes.POINTER(ctypes.c_int)]),
    "gbi_mlp_labels": (_I, [_VP, _I, _D, _VP, _VP, _VP, _VP, c_double_p, _VP]),
    "gbi_mlp_loss_grad": (_I, [_VP, _I, _VP, _VP, _D, _I, ctypes.POINTER(ctypes.c_int), _VP, c_double_p, _VP]),
    "gbi_mlp_adam": (_I, [_VP, _VP, _D]),
    "gbi_mlp_train": (_I, [_VP, _I, _VP, _VP, _D, _I, ctypes.POINTER(ctypes.c_int), _VP, _I, _I, _D, _D,
                           c_double_p]),
    "gbi_mlp_set_head": (_I, [_VP, _I]),
    "gbi_mlp_correct_qh": (_I, [_VP, _I, _VP, _VP, _D, _D, _I, ctypes.POINTER(ctypes.c_int), _I, _VP,
                                ctypes.POINTER(ctypes.c_int)]),
    "gbi_mlp_labels_qh": (_I, [_VP, _I, _I, _D, _VP, _VP, c_double_p, _VP]),
    "gbi_qh_onebody": (_I, [_VP, ctypes.POINTER(gbi_params), _I, _VP, _VP]),
    "gbi_wall_superpose": (_I, [_VP, ctypes.POINTER(gbi_params), _I] + [_VP] * 8),
    "gbi_periodic_superpose": (_I, [_VP, ctypes.POINTER(gbi_params), _I, _D, _VP, _VP, _VP, _VP,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), c_double_p,
                                    ctypes.POINTER(ctypes.c_longlong)]),
    "gbi_kernel_launches": (ctypes.c_longlong, [_VP]),
    "gbi_solve_graph_replays": (ctypes.c_longlong, [_VP]),
    "gbi_set_profiling": (_I, [_VP, _I]),
    "gbi_kernel_stats": (_I, [_VP, _I, c_double_p, ctypes.POINTER(ctypes.c_longlong), c_double_p]),
}

# kernel classes of gbi_kernel_stats
def kernel_class(precision, rows, cols):
    return precision * 9 + rows * 3 + cols


TRAP_F64, TRAP_F32 = 27, 28
FLOW_F64, FLOW_F32 = 29, 30
WALL_F64, WALL_F32 = 31, 32
MLP_NPARAM = 35078
N_KERNEL_CLASSES = 33


def lib():
    """Load libgbi.so (built in-tree by ``paper_1411_0278_gb300.build``)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libgbi.so is not built (%s); run paper_1411_0278_gb300.build.build() "
                              "on a machine with nvcc -- there is no CPU fallback" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def status_string(status):
    return lib().gbi_status_string(int(status)).decode()


def h(trunc):
    return lib().gbi_h(int(trunc))


def d(trunc):
    return lib().gbi_d(int(trunc))


def _host_table(fn, trunc):
    n = d(trunc)
    if n < 0:
        raise GbiError(GBI_ERR_ARG, fn)
    buf = (ctypes.c_double * n)()
    st = getattr(lib(), fn)(int(trunc), buf)
    if st != GBI_OK:
        raise GbiError(st, fn)
    return list(buf)


def component_scales(trunc):
    return _host_table("gbi_component_scales", trunc)


def self_scalars(trunc):
    return _host_table("gbi_self_scalars", trunc)


def _ptr(t, dtype=None):
    """Device address of a contiguous CUDA tensor of the expected dtype (float64 unless given)."""
    if t is None or t.numel() == 0:
        return None
    import torch
    dtype = torch.float64 if dtype is None else dtype
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError("expected a contiguous %s CUDA tensor" % dtype)
    return ctypes.c_void_p(t.data_ptr())


def _f32(t):
    import torch
    return _ptr(t, torch.float32)


def _i32(t):
    import torch
    return _ptr(t, torch.int32)


def solve_static(prm, R, Va, Oa, VH, Fe, Te, V, Om, QH, warm_start=False, stream=None):
    """gbi_solve_static: the solve with all scratch in the library's static device array.

    Outputs V, Om, QH are caller-allocated float64 CUDA tensors; returns (info, status)."""
    info = gbi_info()
    handle = getattr(stream, "cuda_stream", stream)
    st = lib().gbi_solve_static(ctypes.c_void_p(int(handle) if handle else 0), ctypes.byref(prm), int(R.shape[0]),
                                _ptr(R), _ptr(Va), _ptr(Oa), _ptr(VH), _ptr(Fe), _ptr(Te), _ptr(V), _ptr(Om),
                                _ptr(QH), int(bool(warm_start)), ctypes.byref(info))
    if st not in (GBI_OK, GBI_ERR_NOT_CONVERGED):
        raise GbiError(st, "gbi_solve_static")
    return info, st


def params(a=1.0, eta=1.0, trunc=2, precision=1, rtol=1e-10, restart=40, max_iter=1000, max_refine=8,
           inner_rtol=1e-5, min_sep=0.0):
    return gbi_params(float(a), float(eta), int(trunc), int(precision), float(rtol), int(restart),
                      int(max_iter), int(max_refine), float(inner_rtol), float(min_sep))


class Context:
    """gbi_create / gbi_destroy; bound to one device and (optionally) a torch stream."""

    def __init__(self, device=0, stream=None):
        self._h = ctypes.c_void_p()
        st = lib().gbi_create(ctypes.byref(self._h), int(device))
        if st != GBI_OK:
            raise GbiError(st, "gbi_create")
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        self._check(lib().gbi_set_stream(self._h, ctypes.c_void_p(int(handle) if handle else 0)), "gbi_set_stream")

    def synchronize(self):
        self._check(lib().gbi_synchronize(self._h), "gbi_synchronize")

    def close(self):
        if self._h:
            lib().gbi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, where, allow=()):
        if st != GBI_OK and st not in allow:
            raise GbiError(st, where, lib().gbi_last_error(self._h).decode())
        return st

    # ------------------------------------------------------------------ calls

    def apply(self, N, trunc, a, rows, cols, precision, R, x, y, alpha=1.0, beta=0.0, add_self=False):
        return self._check(lib().gbi_apply(self._h, int(N), int(trunc), float(a), int(rows), int(cols),
                                           int(precision), _ptr(R), _ptr(x), _ptr(y), float(alpha), float(beta),
                                           int(bool(add_self))), "gbi_apply")

    def solve(self, prm, R, Va, Oa, VH, Fe, Te, QH=None, warm_start=False, allow_not_converged=False):
        import torch
        N = R.shape[0]
        V = torch.empty((N, 3), dtype=torch.float64, device=R.device)
        Om = torch.empty_like(V)
        if QH is None:
            QH = torch.zeros((N, max(h(prm.trunc), 0)), dtype=torch.float64, device=R.device)
        info = gbi_info()
        st = lib().gbi_solve(self._h, ctypes.byref(prm), int(N), _ptr(R), _ptr(Va), _ptr(Oa), _ptr(VH), _ptr(Fe),
                             _ptr(Te), _ptr(V), _ptr(Om), _ptr(QH), int(bool(warm_start)), ctypes.byref(info))
        self._check(st, "gbi_solve", allow=(GBI_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return V, Om, QH, info, st

    def batch_solve(self, prm, offsets, R, Va, Oa, VH, Fe, Te, QH=None, warm_start=False,
                    allow_not_converged=False):
        """gbi_batch_solve: offsets is a host sequence of nsys + 1 sphere offsets."""
        import torch
        N = R.shape[0]
        offs = (ctypes.c_int * len(offsets))(*[int(o) for o in offsets])
        V = torch.empty((N, 3), dtype=torch.float64, device=R.device)
        Om = torch.empty_like(V)
        if QH is None:
            QH = torch.zeros((N, max(h(prm.trunc), 0)), dtype=torch.float64, device=R.device)
        info = gbi_info()
        st = lib().gbi_batch_solve(self._h, ctypes.byref(prm), len(offsets) - 1, offs, _ptr(R), _ptr(Va), _ptr(Oa),
                                   _ptr(VH), _ptr(Fe), _ptr(Te), _ptr(V), _ptr(Om), _ptr(QH),
                                   int(bool(warm_start)), ctypes.byref(info))
        self._check(st, "gbi_batch_solve", allow=(GBI_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return V, Om, QH, info, st

    def solve_host(self, prm, R, Va, Oa, VH, Fe, Te, V, Om, QH, warm_start=False):
        """Host-memory variant: arguments are C-contiguous float64 numpy arrays (pinned or not)."""
        def p(a):
            return ctypes.c_void_p(a.ctypes.data) if a is not None else None
        info = gbi_info()
        st = lib().gbi_solve_host(self._h, ctypes.byref(prm), int(R.shape[0]), p(R), p(Va), p(Oa), p(VH), p(Fe),
                                  p(Te), p(V), p(Om), p(QH), int(bool(warm_start)), ctypes.byref(info))
        self._check(st, "gbi_solve_host", allow=(GBI_ERR_NOT_CONVERGED,))
        return info, st

    def solve_host_ptrs(self, prm, N, ptrs, warm_start=False):
        """Host-memory variant taking raw addresses (e.g. pinned torch tensors' data_ptr())."""
        info = gbi_info()
        st = lib().gbi_solve_host(self._h, ctypes.byref(prm), int(N), *[ctypes.c_void_p(p) for p in ptrs],
                                  int(bool(warm_start)), ctypes.byref(info))
        self._check(st, "gbi_solve_host", allow=(GBI_ERR_NOT_CONVERGED,))
        return info, st

    def superpose(self, prm, R, Va, Oa, VH, Fe, Te, V=None, Om=None):
        import torch
        N = R.shape[0]
        V = torch.empty((N, 3), dtype=torch.float64, device=R.device) if V is None else V
        Om = torch.empty_like(V) if Om is None else Om
        self._check(lib().gbi_superpose(self._h, ctypes.byref(prm), int(N), _ptr(R), _ptr(Va), _ptr(Oa), _ptr(VH),
                                        _ptr(Fe), _ptr(Te), _ptr(V), _ptr(Om)), "gbi_superpose")
        return V, Om

    def batch_superpose(self, prm, offsets, R, Va, Oa, VH, Fe, Te, V=None, Om=None):
        """gbi_batch_superpose: superposition velocities of independent suspensions."""
        import torch
        N = R.shape[0]
        offs = (ctypes.c_int * len(offsets))(*[int(o) for o in offsets])
        V = torch.empty((N, 3), dtype=torch.float64, device=R.device) if V is None else V
        Om = torch.empty_like(V) if Om is None else Om
        self._check(lib().gbi_batch_superpose(self._h, ctypes.byref(prm), len(offsets) - 1, offs, _ptr(R), _ptr(Va),
                                              _ptr(Oa), _ptr(VH), _ptr(Fe), _ptr(Te), _ptr(V), _ptr(Om)),
                    "gbi_batch_superpose")
        return V, Om

    def trap_inputs(self, N, trunc, k_trap, vs, s0, d0, R, p):
        import torch
        dev = R.device
        out = [torch.empty((N, 3), dtype=torch.float64, device=dev) for _ in range(4)]
        VH = torch.empty((N, h(trunc)), dtype=torch.float64, device=dev)
        self._check(lib().gbi_trap_inputs(self._h, int(N), int(trunc), float(k_trap), float(vs), float(s0),
                                          float(d0), _ptr(R), _ptr(p), *[_ptr(t) for t in out], _ptr(VH)),
                    "gbi_trap_inputs")
        Fe, Te, Va, Oa = out
        return dict(Fe=Fe, Te=Te, Va=Va, Oa=Oa, VH=VH)

    def tune(self, trunc, offsets, reps=0):
        """gbi_tune: time each warps-per-target choice of the pair passes on synthetic
        input with the sphere layout ``offsets`` (nsys + 1 ints); returns the 6 choices
        (H/H FP32, H/H double-float, H/L and L/all double-float, H/L and L/all FP32)."""
        off = (ctypes.c_int * len(offsets))(*[int(v) for v in offsets])
        out = (ctypes.c_int * 6)()
        self._check(lib().gbi_tune(self._h, int(trunc), len(offsets) - 1, off, int(reps), out), "gbi_tune")
        return list(out)

    def set_wpt(self, wpt):
        self._check(lib().gbi_set_wpt(self._h, int(wpt)), "gbi_set_wpt")

    def set_split_tail(self, on):
        self._check(lib().gbi_set_split_tail(self._h, int(on)), "gbi_set_split_tail")

    def set_wait_limit(self, rounds):
        self._check(lib().gbi_set_wait_limit(self._h, int(rounds)), "gbi_set_wait_limit")

    def pass_status(self):
        """gbi_pass_status: the status code (GBI_OK or GBI_ERR_TIMEOUT), not raised."""
        return lib().gbi_pass_status(self._h)

    def pass_wpt(self, trunc, rows, cols, precision, N, batched=False):
        return lib().gbi_pass_wpt(self._h, int(trunc), int(rows), int(cols), int(precision), int(N), int(batched))

    # ---- learned near-field correction
    @staticmethod
    def _offs(offsets):
        if offsets is None:
            return 0, None
        return len(offsets) - 1, (ctypes.c_int * len(offsets))(*[int(v) for v in offsets])

    def pairs(self, R, a, rcut, offsets=None):
        """gbi_pairs + gbi_pairs_get: (targets, sources) int32 device tensors."""
        import torch
        nsys, offs = self._offs(offsets)
        n = ctypes.c_int()
        self._check(lib().gbi_pairs(self._h, int(R.shape[0]), _ptr(R), float(a), float(rcut), nsys, offs,
                                    ctypes.byref(n)), "gbi_pairs")
        tg = torch.empty(n.value, dtype=torch.int32, device=R.device)
        sr = torch.empty_like(tg)
        self._check(lib().gbi_pairs_get(self._h, _i32(tg), _i32(sr)), "gbi_pairs_get")
        return tg, sr

    def mlp_set(self, theta, sigma):
        import numpy as np
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == MLP_NPARAM
        self._check(lib().gbi_mlp_set(self._h, th.ctypes.data, float(sigma)), "gbi_mlp_set")

    def mlp_get(self):
        import numpy as np
        th = np.empty(MLP_NPARAM, dtype=np.float32)
        sig = ctypes.c_double()
        self._check(lib().gbi_mlp_get(self._h, th.ctypes.data, ctypes.byref(sig)), "gbi_mlp_get")
        return th, sig.value

    def mlp_features(self, R, p, tg, sr, a):
        import torch
        P = int(tg.shape[0])
        F = torch.empty((P, 9), dtype=torch.float32, device=R.device)
        FR = torch.empty((P, 9), dtype=torch.float32, device=R.device)
        self._check(lib().gbi_mlp_features(self._h, P, _ptr(R), _ptr(p), _i32(tg), _i32(sr), float(a), _f32(F),
                                           _f32(FR)), "gbi_mlp_features")
        return F, FR

    def mlp_forward(self, F, FR=None):
        import torch
        P = int(F.shape[0])
        out = torch.empty((P, 6), dtype=torch.float32, device=F.device)
        self._check(lib().gbi_mlp_forward(self._h, P, _f32(F), _f32(FR) if FR is not None else None, _f32(out)),
                    "gbi_mlp_forward")
        return out

    def mlp_set_engine(self, engine):
        """0: mma.sync inference kernel, 1: tcgen05 (tensor memory) inference kernel."""
        self._check(lib().gbi_mlp_set_engine(self._h, int(engine)), "gbi_mlp_set_engine")

    def mlp_status(self):
        """gbi_mlp_status: raises GbiError if a tensor-core completion wait gave up."""
        self._check(lib().gbi_mlp_status(self._h), "gbi_mlp_status")

    def mlp_correct(self, R, p, a, s0, V, Om, offsets=None):
        nsys, offs = self._offs(offsets)
        n = ctypes.c_int()
        self._check(lib().gbi_mlp_correct(self._h, int(R.shape[0]), _ptr(R), _ptr(p), float(a), float(s0), nsys,
                                          offs, _ptr(V), _ptr(Om), ctypes.byref(n)), "gbi_mlp_correct")
        return n.value

    def mlp_labels(self, s0, Vx, Ox, Vs, Os, sigma=0.0):
        import torch
        N = int(Vx.shape[0])
        lab = torch.empty((N, 6), dtype=torch.float64, device=Vx.device)
        sig = ctypes.c_double(float(sigma))
        self._check(lib().gbi_mlp_labels(self._h, N, float(s0), _ptr(Vx), _ptr(Ox), _ptr(Vs), _ptr(Os),
                                         ctypes.byref(sig), _ptr(lab)), "gbi_mlp_labels")
        return lab, sig.value

    def mlp_set_head(self, head):
        """0: velocity-correction head, 1: strain-mode Q^(2s) head (warm start of the solve)."""
        self._check(lib().gbi_mlp_set_head(self._h, int(head)), "gbi_mlp_set_head")

    def mlp_correct_qh(self, R, p, a, s0, QH, offsets=None):
        nsys, offs = self._offs(offsets)
        n = ctypes.c_int()
        self._check(lib().gbi_mlp_correct_qh(self._h, int(R.shape[0]), _ptr(R), _ptr(p), float(a), float(s0), nsys,
                                             offs, int(QH.shape[1]), _ptr(QH), ctypes.byref(n)), "gbi_mlp_correct_qh")
        return n.value

    def mlp_labels_qh(self, s0, QHx, QH1, sigma=0.0):
        import torch
        N = int(QHx.shape[0])
        lab = torch.empty((N, 6), dtype=torch.float64, device=QHx.device)
        sig = ctypes.c_double(float(sigma))
        self._check(lib().gbi_mlp_labels_qh(self._h, N, int(QHx.shape[1]), float(s0), _ptr(QHx), _ptr(QH1),
                                            ctypes.byref(sig), _ptr(lab)), "gbi_mlp_labels_qh")
        return lab, sig.value

    def wall_superpose(self, prm, R, Va, Oa, VH, Fe, Te, V=None, Om=None):
        """gbi_wall_superpose: superposition above the wall z = 0 (outputs allocated if None)."""
        import torch
        N = R.shape[0]
        if V is None:
            V = torch.empty((N, 3), dtype=torch.float64, device=R.device)
        if Om is None:
            Om = torch.empty_like(V)
        self._check(lib().gbi_wall_superpose(self._h, ctypes.byref(prm), int(N), _ptr(R), _ptr(Va), _ptr(Oa),
                                             _ptr(VH), _ptr(Fe), _ptr(Te), _ptr(V), _ptr(Om)), "gbi_wall_superpose")
        return V, Om

    def periodic_superpose(self, prm, L, R, Va, Fe, V=None, cells=0, mesh=0):
        """gbi_periodic_superpose: point-force superposition in the periodic cube of side L
        (cells: 0 choose, >= 3 impose, < 0 every pair; mesh: 0 choose, a power of 2 in
        [16, 512] impose, < 0 the direct wave-space sum).  Returns (V, plan) with
        plan = dict(cells_per_side, mesh, xi, n_wave)."""
        import torch
        N = R.shape[0]
        if V is None:
            V = torch.empty((N, 3), dtype=torch.float64, device=R.device)
        M = ctypes.c_int(int(cells))
        K = ctypes.c_int(int(mesh))
        xi = ctypes.c_double()
        nk = ctypes.c_longlong()
        self._check(lib().gbi_periodic_superpose(self._h, ctypes.byref(prm), int(N), float(L), _ptr(R), _ptr(Va),
                                                 _ptr(Fe), _ptr(V), ctypes.byref(M), ctypes.byref(K),
                                                 ctypes.byref(xi), ctypes.byref(nk)), "gbi_periodic_superpose")
        return V, dict(cells_per_side=M.value, mesh=K.value, xi=xi.value, n_wave=nk.value)

    def qh_onebody(self, prm, VH):
        import torch
        QH = torch.empty_like(VH)
        self._check(lib().gbi_qh_onebody(self._h, ctypes.byref(prm), int(VH.shape[0]), _ptr(VH), _ptr(QH)),
                    "gbi_qh_onebody")
        return QH

    def mlp_loss_grad(self, R, p, a, labels, offsets=None):
        import torch
        nsys, offs = self._offs(offsets)
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=R.device)
        loss = ctypes.c_double()
        self._check(lib().gbi_mlp_loss_grad(self._h, int(R.shape[0]), _ptr(R), _ptr(p), float(a), nsys, offs,
                                            _ptr(labels), ctypes.byref(loss), _f32(g)), "gbi_mlp_loss_grad")
        return loss.value, g

    def mlp_adam(self, grad, lr):
        self._check(lib().gbi_mlp_adam(self._h, _f32(grad), float(lr)), "gbi_mlp_adam")

    def mlp_train(self, R, p, a, offsets, labels, epochs, batch_systems, lr0, lr1):
        nsys, offs = self._offs(offsets)
        hist = (ctypes.c_double * max(int(epochs), 1))()
        self._check(lib().gbi_mlp_train(self._h, int(R.shape[0]), _ptr(R), _ptr(p), float(a), nsys, offs,
                                        _ptr(labels), int(epochs), int(batch_systems), float(lr0), float(lr1), hist),
                    "gbi_mlp_train")
        return list(hist)[:int(epochs)]

    def kernel_launches(self):
        return int(lib().gbi_kernel_launches(self._h))

    def solve_graph_replays(self):
        return int(lib().gbi_solve_graph_replays(self._h))

    def set_profiling(self, on):
        self._check(lib().gbi_set_profiling(self._h, int(bool(on))), "gbi_set_profiling")

    def kernel_stats(self, cls):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        fl = ctypes.c_double()
        self._check(lib().gbi_kernel_stats(self._h, int(cls), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl)),
                    "gbi_kernel_stats")
        return dict(ms=ms.value, launches=n.value, flops=fl.value)

    def squirmer_inputs(self, N, trunc, k_trap, B1, B2, R, p):
        import torch
        z = lambda *shape: torch.empty(shape, dtype=torch.float64, device=R.device)
        out = dict(Fe=z(N, 3), Te=z(N, 3), Va=z(N, 3), Oa=z(N, 3), VH=z(N, max(h(trunc), 1)))
        self._check(lib().gbi_squirmer_inputs(self._h, int(N), int(trunc), float(k_trap), float(B1), float(B2),
                                              _ptr(R), _ptr(p), _ptr(out["Fe"]), _ptr(out["Te"]), _ptr(out["Va"]),
                                              _ptr(out["Oa"]), _ptr(out["VH"])), "gbi_squirmer_inputs")
        return out

    def squirmer_step(self, prm, R, p, dt, k_trap, B1, B2, superposition, nsteps):
        info = gbi_info()
        st = lib().gbi_squirmer_step(self._h, ctypes.byref(prm), int(R.shape[0]), float(dt), float(k_trap),
                                     float(B1), float(B2), int(bool(superposition)), int(nsteps), _ptr(R), _ptr(p),
                                     ctypes.byref(info))
        self._check(st, "gbi_squirmer_step")
        return info

    def flow(self, prm, R, Fe, Te, QH, X, U=None):
        """gbi_flow: the flow at points X [M][3] of a solved suspension; returns (U, inside count)."""
        import torch
        M = X.shape[0]
        if U is None:
            U = torch.empty((M, 3), dtype=torch.float64, device=X.device)
        n_in = ctypes.c_int(0)
        N = R.shape[0]
        self._check(lib().gbi_flow(self._h, ctypes.byref(prm), int(N), _ptr(R), _ptr(Fe), _ptr(Te), _ptr(QH),
                                   int(M), _ptr(X), _ptr(U), ctypes.byref(n_in)), "gbi_flow")
        return U, n_in.value

    def batch_trap_step(self, prm, offsets, R, p, dt, k_trap, vs, s0, d0, superposition, nsteps):
        info = gbi_info()
        nsys, off = self._offs(offsets)
        st = lib().gbi_batch_trap_step(self._h, ctypes.byref(prm), nsys, off, float(dt), float(k_trap),
                                       float(vs), float(s0), float(d0), int(bool(superposition)), int(nsteps),
                                       _ptr(R), _ptr(p), ctypes.byref(info))
        self._check(st, "gbi_batch_trap_step")
        return info

    def trap_step(self, prm, R, p, dt, k_trap, vs, s0, d0, superposition, nsteps):
        info = gbi_info()
        st = lib().gbi_trap_step(self._h, ctypes.byref(prm), int(R.shape[0]), float(dt), float(k_trap), float(vs),
                                 float(s0), float(d0), int(bool(superposition)), int(nsteps), _ptr(R), _ptr(p),
                                 ctypes.byref(info))
        self._check(st, "gbi_trap_step")
        return info
