"""ctypes binding of libmg.so (include/mg.h): argument marshalling only.

Every step of the solve runs inside the CUDA library.  Arrays may be torch
tensors (CUDA or CPU) or numpy arrays; they must be C-contiguous with the
dtype the call expects.  Importing this module does not need a GPU; loading
the library does need the built libmg.so and fails loudly without it.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmg.so")

MG_OK = 0
STATUS_NAMES = {0: "MG_OK", 1: "MG_ERR_INVALID_ARG", 2: "MG_ERR_OOM", 3: "MG_ERR_CUDA",
                4: "MG_ERR_NOT_CONVERGED", 5: "MG_ERR_TIMEOUT", 6: "MG_ERR_NO_WEIGHTS",
                7: "MG_ERR_BAD_WEIGHTS", 8: "MG_ERR_NONFINITE"}
PROLONG = {"cubic": 0, "sr": 1}
PRECISION = {"fp64": 0, "mixed": 1}

# every exported symbol and its signature (restype, argtypes)
_VP, _I, _D, _SZ = C.c_void_p, C.c_int, C.c_double, C.c_size_t


class SolveInfo(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("vcycles", C.c_int), ("rel_residual", C.c_double),
                ("removed_mean", C.c_double), ("update_norm", C.c_double), ("time_ms", C.c_double),
                ("prolong_used", C.c_int), ("sr_fallback", C.c_int), ("sr_cycles", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerResult(C.Structure):
    _fields_ = [("request_id", C.c_longlong), ("stream_id", C.c_int), ("N", C.c_int), ("status", C.c_int),
                ("pad", C.c_int), ("t_submit_ms", C.c_double), ("t_admit_ms", C.c_double),
                ("t_finish_ms", C.c_double), ("info", SolveInfo)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("pad", "info")}
        d.update(self.info.as_dict())
        return d


SIGNATURES = {
    "mg_setup": (_I, [_I, _I, C.POINTER(_VP)]),
    "mg_set_options": (_I, [_VP, _I, _I, _I, _I, _VP]),
    "mg_set_inner_cycles": (_I, [_VP, _I]),
    "mg_set_adaptive_cycles": (_I, [_VP, _I, _D]),
    "mg_set_graph_execution": (_I, [_VP, _I]),
    "mg_set_prolong_policy": (_I, [_VP, _D, _D]),
    "mg_load_prolong_weights": (_I, [_VP, _VP, _SZ]),
    "mg_solve": (_I, [_VP, _VP, _VP, _D, _I, C.POINTER(SolveInfo)]),
    "mg_vcycle": (_I, [_VP, _VP, _VP, _I]),
    "mg_two_level_solve": (_I, [_VP, _VP, _VP, _D, _I, _I, _I, _I, _I, C.POINTER(SolveInfo)]),
    "mg_solve_batched": (_I, [C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP), _I, _D, _I,
                              C.POINTER(SolveInfo)]),
    "mg_destroy": (None, [_VP]),
    "mg_autotune": (_I, [_VP, C.c_char_p, C.POINTER(_I)]),
    "mg_get_tile_variant": (_I, [_I, _I, _I, C.POINTER(_I)]),
    "mg_set_launch_overlap": (_I, [_I]),
    "mg_get_launch_overlap": (_I, []),
    "mg_set_tile_variant": (_I, [_I, _I, _I, _I]),
    "mg_server_create": (_I, [_SZ, _I, _I, _I, _I, _D, _VP, C.POINTER(_VP)]),
    "mg_server_submit": (_I, [_VP, _I, _I, _VP, _VP, C.POINTER(C.c_longlong)]),
    "mg_server_tick": (_I, [_VP, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "mg_server_poll": (_I, [_VP, C.POINTER(ServerResult), C.POINTER(_I)]),
    "mg_server_destroy": (None, [_VP]),
    "mg_trainer_create": (_I, [_I, _I, _I, _VP, _SZ, _D, C.POINTER(_VP)]),
    "mg_trainer_forward": (_I, [_VP, _VP, _VP]),
    "mg_trainer_gradients": (_I, [_VP, _VP, _VP, _VP, _VP, C.POINTER(_D)]),
    "mg_trainer_step": (_I, [_VP, _VP, _VP, _VP, C.POINTER(_D)]),
    "mg_trainer_set_lr": (_I, [_VP, _D]),
    "mg_trainer_set_tensor_cores": (_I, [_VP, _I]),
    "mg_set_tma_tiles": (_I, [_I]),
    "mg_set_zero_guess": (_I, [_VP, _I]),
    "mg_set_coarse_cluster": (_I, [_I]),
    "mg_get_coarse_cluster": (_I, []),
    "mg_set_fused_update": (_I, [_I]),
    "mg_get_fused_update": (_I, []),
    "mg_set_fp64_separate_x_pass": (_I, [_I]),
    "mg_get_fp64_separate_x_pass": (_I, []),
    "mg_get_tma_tiles": (_I, []),
    "mg_trainer_get_tensor_cores": (_I, [_VP, C.POINTER(_I)]),
    "mg_trainer_get_weights": (_I, [_VP, _VP, _SZ]),
    "mg_trainer_destroy": (None, [_VP]),
    "mg_status_string": (C.c_char_p, [_I]),
    "mg_last_error": (C.c_char_p, []),
    "mg_kernel_launches": (C.c_ulonglong, []),
    "mg_probe_kernel": (_I, [_VP, _I, _I]),
    "mg_probe_read": (_I, [_VP, C.POINTER(_I), C.POINTER(_D), C.POINTER(_D)]),
    "mg_op_down": (_I, [_I, _I, _VP, _VP, _VP, _I, _I, _VP, _VP]),
    "mg_op_up": (_I, [_I, _I, _VP, _VP, _VP, _VP, _I, _VP]),
    "mg_op_vcycle": (_I, [_I, _I, _I, _VP, _VP, _I, _I, _I, _VP]),
    "mg_op_vcycle_static": (_I, [_I, _I, _I, _VP, _VP, _I, _I, _I, _VP]),
    "mg_op_sr_conv": (_I, [_I, _I, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "mg_op_sr_generator": (_I, [_VP, _VP, _I, _VP]),
    "mg_op_sr_layer": (_I, [_VP, _I, _I, _VP, _VP, _VP, _VP]),
    "mg_op_sr_windowed": (_I, [_VP, _VP, _I, _D, _D, _VP]),
    "mg_op_outer_residual": (_I, [_I, _VP, _VP, _D, _VP, _VP, _VP]),
    "mg_op_convert": (_I, [_I, _SZ, _VP, _VP, _VP]),
}

_lib = None


class MGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libmg.so once.  Raises if the library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_2403_07936_gb300.build.build() "
                          "(the CUDA library is required; there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != MG_OK:
        raise MGError(status, load().mg_last_error().decode(errors="replace"))


def ptr(a) -> int:
    """Raw address of a contiguous torch tensor or numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def stream_handle(stream) -> int | None:
    """cudaStream_t of a torch.cuda.Stream (or an int handle, or None)."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_code(a) -> int:
    name = str(a.dtype)
    if "float64" in name:
        return 0
    if "float32" in name:
        return 1
    raise TypeError(f"dtype {a.dtype} not supported (float64 or float32)")


@dataclass
class Options:
    precision: str = "mixed"
    nu_pre: int = 2
    nu_post: int = 2
    max_cycles: int = 100
    inner_cycles: int = 2


class Context:
    """A solver context for N x N grids with `levels` levels (mg_setup)."""

    def __init__(self, levels: int, N: int, **opts):
        lib = load()
        h = C.c_void_p()
        _check(lib.mg_setup(levels, N, C.byref(h)))
        self._h = h
        self.N = N
        self.levels = levels
        self.options = Options()
        self._stream = None
        if opts:
            self.set_options(**opts)

    @property
    def handle(self):
        return self._h

    def set_options(self, precision=None, nu_pre=None, nu_post=None, max_cycles=None,
                    inner_cycles=None, stream="keep"):
        o = self.options
        if precision is not None:
            o.precision = precision
        if nu_pre is not None:
            o.nu_pre = nu_pre
        if nu_post is not None:
            o.nu_post = nu_post
        if max_cycles is not None:
            o.max_cycles = max_cycles
        if stream != "keep":
            self._stream = stream_handle(stream)
        lib = load()
        _check(lib.mg_set_options(self._h, PRECISION[o.precision], o.nu_pre, o.nu_post,
                                  o.max_cycles, self._stream))
        if inner_cycles is not None:
            o.inner_cycles = inner_cycles
            _check(lib.mg_set_inner_cycles(self._h, inner_cycles))

    def set_adaptive_cycles(self, m_max: int = 3, rho: float = 0.06):
        """Adaptive V-cycles per outer step (mg_set_adaptive_cycles); rho = 0 turns it off."""
        _check(load().mg_set_adaptive_cycles(self._h, m_max, rho))

    def set_prolong_policy(self, n_gan: float = float("inf"), s_thres: float = 0.0):
        """Hybrid SR / cubic choice per V-cycle for prolong="sr" solves (mg_set_prolong_policy)."""
        _check(load().mg_set_prolong_policy(self._h, n_gan, s_thres))

    def set_graph_execution(self, enable: bool):
        """Run mg_solve as one CUDA graph launch (True, default) or a host loop."""
        _check(load().mg_set_graph_execution(self._h, int(bool(enable))))

    def load_weights(self, blob: bytes):
        buf = C.create_string_buffer(bytes(blob), len(blob))
        _check(load().mg_load_prolong_weights(self._h, C.cast(buf, C.c_void_p), len(blob)))

    def solve(self, f, x, tol: float = 1e-10, prolong: str = "cubic", check: bool = True) -> dict:
        info = SolveInfo()
        st = load().mg_solve(self._h, ptr(f), ptr(x), tol, PROLONG[prolong], C.byref(info))
        d = info.as_dict()
        d["status"] = STATUS_NAMES.get(st, st)
        if check and st != MG_OK:
            _check(st)
        return d

    def set_zero_guess(self, on: bool):
        """Solves start from x = 0 and never read x (no host-to-device copy of a host x)."""
        _check(load().mg_set_zero_guess(self._h, int(bool(on))))

    def vcycle(self, f, x, prolong: str = "cubic"):
        _check(load().mg_vcycle(self._h, ptr(f), ptr(x), PROLONG[prolong]))

    def two_level_solve(self, f, x, tol: float = 1e-10, coarsen_log2: int = 4, nu_smooth: int = 20,
                        coarse_sweeps: int = 10, max_cycles: int = 300, prolong: str = "cubic",
                        check: bool = True) -> dict:
        """The paper's two-level configuration (mg_two_level_solve): one coarse
        level 2^coarsen_log2 times coarser, nu_smooth fine sweeps, coarse_sweeps
        coarse sweeps, prolongation by 2^coarsen_log2 with the cubic spline or
        ("sr") the generator applied once per factor 2."""
        info = SolveInfo()
        st = load().mg_two_level_solve(self._h, ptr(f), ptr(x), tol, coarsen_log2, nu_smooth, coarse_sweeps,
                                       max_cycles, PROLONG[prolong], C.byref(info))
        d = info.as_dict()
        d["status"] = STATUS_NAMES.get(st, st)
        if check and st not in (MG_OK,):
            _check(st)
        return d

    def autotune(self, cache_path: str | None = None) -> int:
        """Time the tile variants on this context's levels; returns entries measured."""
        n = _I()
        path = cache_path.encode() if cache_path else None
        _check(load().mg_autotune(self._h, path, C.byref(n)))
        return n.value

    def probe(self, kind: int, capacity: int = 256):
        """Time one kernel kind with CUDA events (1 down, 2 up, 3 residual, 4 update, 5 coarse span,
        6 update fused with the next residual)."""
        _check(load().mg_probe_kernel(self._h, kind, capacity))

    def probe_read(self):
        n, ms, by = C.c_int(), C.c_double(), C.c_double()
        _check(load().mg_probe_read(self._h, C.byref(n), C.byref(ms), C.byref(by)))
        return n.value, ms.value, by.value

    def close(self):
        if self._h:
            load().mg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (mg_server_* in include/mg.h).

    submit() queues a request; tick() admits what fits the memory budget, runs
    one outer defect-correction step for every admitted request and retires
    the converged ones; poll() returns retired requests.  The caller keeps f
    (and x_out) alive until the request has retired.  inner_cycles = 0 (the
    default) picks each request's V-cycles per step adaptively from its own
    residual history.
    """

    def __init__(self, hbm_budget_bytes: int, nu_pre: int = 2, nu_post: int = 2, inner_cycles: int = 0,
                 max_cycles: int = 100, tol: float = 1e-10, stream=None):
        h = C.c_void_p()
        _check(load().mg_server_create(int(hbm_budget_bytes), nu_pre, nu_post, inner_cycles, max_cycles, tol,
                                       stream_handle(stream), C.byref(h)))
        self._h = h

    def submit(self, f, x_out=None, stream_id: int = -1) -> int:
        rid = C.c_longlong()
        _check(load().mg_server_submit(self._h, stream_id, f.shape[-1], ptr(f), ptr(x_out), C.byref(rid)))
        return rid.value

    def tick(self):
        a, q, d = _I(), _I(), _I()
        _check(load().mg_server_tick(self._h, C.byref(a), C.byref(q), C.byref(d)))
        return a.value, q.value, d.value

    def poll(self):
        """All retired requests not yet returned, as dicts."""
        out = []
        r, got = ServerResult(), _I()
        while True:
            _check(load().mg_server_poll(self._h, C.byref(r), C.byref(got)))
            if not got.value:
                return out
            out.append(r.as_dict())

    def close(self):
        if self._h:
            load().mg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_launch_overlap(mode):
    """Programmatic dependent launch between library kernels: 0 / False off,
    1 / True every kernel, 2 kernels of grids of at most one wave."""
    _check(load().mg_set_launch_overlap(int(mode)))


def set_coarse_cluster(on: bool):
    """Run a single solve's 128^2 level and bottom V-cycle as one 8-CTA cluster launch (True) or three launches."""
    _check(load().mg_set_coarse_cluster(int(bool(on))))


def get_coarse_cluster() -> bool:
    return bool(load().mg_get_coarse_cluster())


def set_fused_update(on: bool):
    """Fuse each outer step's FP64 update with the next outer residual (True) or launch them apart."""
    _check(load().mg_set_fused_update(int(bool(on))))


def get_fused_update() -> bool:
    return bool(load().mg_get_fused_update())


def set_fp64_separate_x_pass(on: bool):
    """FP64 V-cycles: refine each level's coarse error along x once (True) or inside every up-pass tile."""
    _check(load().mg_set_fp64_separate_x_pass(int(bool(on))))


def get_fp64_separate_x_pass() -> bool:
    return bool(load().mg_get_fp64_separate_x_pass())


def set_tma_tiles(on: bool):
    """Stage the smoother's interior 64-row FP32 tiles by TMA (True) or 16-byte vector loads."""
    _check(load().mg_set_tma_tiles(int(bool(on))))


def get_tma_tiles() -> bool:
    return bool(load().mg_get_tma_tiles())


def get_launch_overlap() -> int:
    return int(load().mg_get_launch_overlap())


def get_tile_variant(kind: int, n: int, nu: int) -> int:
    v = _I()
    _check(load().mg_get_tile_variant(kind, n, nu, C.byref(v)))
    return v.value


def set_tile_variant(kind: int, n: int, nu: int, variant: int):
    _check(load().mg_set_tile_variant(kind, n, nu, variant))


class Trainer:
    """SR generator trainer (mg_trainer_* in include/mg.h); device float32 arrays."""

    def __init__(self, H: int, W: int, batch: int, blob: bytes, lr: float = 1e-4):
        buf = C.create_string_buffer(bytes(blob), len(blob))
        h = C.c_void_p()
        _check(load().mg_trainer_create(H, W, batch, C.cast(buf, C.c_void_p), len(blob), lr, C.byref(h)))
        self._h, self.nbytes = h, len(blob)

    def forward(self, q, y):
        _check(load().mg_trainer_forward(self._h, ptr(q), ptr(y)))

    def gradients(self, q, target, grad, mask=None) -> float:
        loss = _D()
        _check(load().mg_trainer_gradients(self._h, ptr(q), ptr(target), ptr(mask), ptr(grad), C.byref(loss)))
        return loss.value

    def step(self, q, target, mask=None) -> float:
        loss = _D()
        _check(load().mg_trainer_step(self._h, ptr(q), ptr(target), ptr(mask), C.byref(loss)))
        return loss.value

    def set_lr(self, lr: float):
        _check(load().mg_trainer_set_lr(self._h, lr))

    @property
    def tensor_cores(self) -> bool:
        """True if the 64/256-channel convolutions run on the tcgen05 tensor cores (BF16 operands)."""
        v = _I()
        _check(load().mg_trainer_get_tensor_cores(self._h, C.byref(v)))
        return bool(v.value)

    @tensor_cores.setter
    def tensor_cores(self, on: bool):
        _check(load().mg_trainer_set_tensor_cores(self._h, int(bool(on))))

    def weights(self) -> bytes:
        buf = C.create_string_buffer(self.nbytes)
        _check(load().mg_trainer_get_weights(self._h, C.cast(buf, C.c_void_p), self.nbytes))
        return buf.raw

    def close(self):
        if self._h:
            load().mg_trainer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    """Kernels launched by libmg in this process so far."""
    return int(load().mg_kernel_launches())


def solve_batched(ctxs, fs, xs, tol: float = 1e-10, prolong: str = "cubic"):
    B = len(ctxs)
    H = (C.c_void_p * B)(*[c.handle for c in ctxs])
    F = (C.c_void_p * B)(*[ptr(f) for f in fs])
    X = (C.c_void_p * B)(*[ptr(x) for x in xs])
    infos = (SolveInfo * B)()
    st = load().mg_solve_batched(H, F, X, B, tol, PROLONG[prolong], infos)
    _check(st)
    return [i.as_dict() for i in infos]


# ---- operator-level calls (device arrays) --------------------------------

def op_down(x, x_out, b, bc, nu: int, zero_init: bool = False, stream=None):
    _check(load().mg_op_down(_dtype_code(x), x.shape[-1], ptr(x), ptr(x_out), ptr(b), nu,
                             int(zero_init), ptr(bc), stream_handle(stream)))


def op_up(x, x_out, b, ec, nu: int, stream=None):
    _check(load().mg_op_up(_dtype_code(x), x.shape[-1], ptr(x), ptr(x_out), ptr(b), ptr(ec), nu,
                           stream_handle(stream)))


def op_vcycle(x, b, coarsest: int, nu1: int, nu2: int, zero_init: bool = False, stream=None):
    _check(load().mg_op_vcycle(_dtype_code(x), x.shape[-1], coarsest, ptr(x), ptr(b), nu1, nu2,
                               int(zero_init), stream_handle(stream)))


def op_sr_conv(mode: int, H: int, W: int, inp, skip, w_packed, bias, prelu, out, stream=None):
    _check(load().mg_op_sr_conv(mode, H, W, ptr(inp), ptr(skip), ptr(w_packed), ptr(bias), ptr(prelu),
                                ptr(out), stream_handle(stream)))


def op_sr_generator(ctx: "Context", ec, out):
    _check(load().mg_op_sr_generator(ctx.handle, ptr(ec), ec.shape[-1], ptr(out)))


def op_sr_layer(ctx: "Context", layer: int, nc: int, inp, out, s, skip=None):
    """One layer of the context's generator on caller buffers (see mg_op_sr_layer)."""
    _check(load().mg_op_sr_layer(ctx.handle, layer, nc, ptr(inp), ptr(skip), ptr(s), ptr(out)))


def op_sr_windowed(ctx: "Context", ec, out, p_min: float = 1e-10, p_max: float = 1e-3):
    """Windowed SR prolongation with symmetric-log normalisation (see mg_op_sr_windowed)."""
    _check(load().mg_op_sr_windowed(ctx.handle, ptr(ec), ec.shape[-1], p_min, p_max, ptr(out)))


def op_outer_residual(f, x, mu: float, s32, out, stream=None):
    _check(load().mg_op_outer_residual(f.shape[-1], ptr(f), ptr(x), mu, ptr(s32), ptr(out),
                                       stream_handle(stream)))


def op_convert(inp, out, stream=None):
    """Integer-pipe conversion: double -> float (round to nearest even) or float -> double."""
    direction = 0 if "float64" in str(inp.dtype) else 1
    _check(load().mg_op_convert(direction, inp.numel(), ptr(inp), ptr(out), stream_handle(stream)))
