"""Python binding of libsnac.so (ctypes): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module checks tensor arguments,
builds the C structs of ``include/snac.h`` and forwards device pointers and the current PyTorch
stream. It raises if the library has not been built: there is no other code path.

    from paper_2106_03583_gb300 import snac, inputs
    blocks, f = inputs.config("mb2x2")
    plan = snac.Plan(blocks, precision="fp64")
    p = torch.zeros_like(rhs)
    info = plan.solve(rhs, p, tol=1e-10)      # rhs, p: CUDA float64, [block][z][y][x]
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsnac.so")

SNAC_OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "LAYOUT", -3: "OOM", -4: "CUDA", -5: "NOT_CONVERGED",
          -6: "NONFINITE", -7: "INCOMPATIBLE_RHS", -8: "TIMEOUT"}
_BC = {"D": 0, "N": 1, "P": 2, "B": 3}
_PREC = {"fp64": 0, "mixed": 1}

EXPORTS = ("snac_plan_create", "snac_plan_workspace_bytes", "snac_poisson_solve", "snac_plan_info",
           "snac_plan_mode_cycles", "snac_plan_destroy", "snac_status_string", "snac_last_error_message",
           "snac_apply_operator", "snac_residual", "snac_residual_ff", "snac_forward_transform", "snac_backward_update",
           "snac_mode_operator", "snac_mode_vcycles", "snac_plan_set_profiling", "snac_plan_kernel_stats",
           "snac_plan_reset_stats", "snac_residual_noalloc", "snac_pencil_forward", "snac_pencil_backward_update",
           "snac_pencil_setup", "snac_pencil_residual", "snac_mode_solve", "snac_mode_fix_mean",
           "snac_poisson_solve_batch", "snac_test_wait_timeout",
           "snac_engine_create", "snac_engine_submit", "snac_engine_wait", "snac_engine_get_stats",
           "snac_engine_clock", "snac_engine_destroy", "snac_autotune")


class SnacError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"snac: {self.name} ({status}){': ' + msg if msg else ''}")


class _Block(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int64 * 3), ("hi", ctypes.c_int64 * 3), ("h_dx", ctypes.c_void_p * 3),
                ("bc", (ctypes.c_int32 * 2) * 3), ("nbr", (ctypes.c_int32 * 2) * 3)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("nu1", ctypes.c_int32), ("nu2", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("max_cycles", ctypes.c_int32), ("max_coarse", ctypes.c_int32),
                ("fused", ctypes.c_int32), ("inner_reduction", ctypes.c_double), ("shift", ctypes.c_double),
                ("mode_begin", ctypes.c_int32), ("mode_end", ctypes.c_int32), ("onchip", ctypes.c_int32),
                ("bottom_cells", ctypes.c_int32)]


class _KStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("outer_iters", ctypes.c_int32), ("total_cycles", ctypes.c_int32),
                ("max_mode_cycles", ctypes.c_int32), ("levels", ctypes.c_int32), ("n_modes", ctypes.c_int32),
                ("rel_res", ctypes.c_double), ("rhs_norm", ctypes.c_double), ("removed_mean", ctypes.c_double),
                ("graph_rounds", ctypes.c_int32)]


class _EngineOptions(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_cached_plans", ctypes.c_int32), ("hbm_budget", ctypes.c_uint64),
                ("autotune", ctypes.c_int32), ("max_group", ctypes.c_int32)]


class _Times(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("worker", ctypes.c_int32), ("plan_reused", ctypes.c_int32),
                ("tuned", ctypes.c_int32), ("group", ctypes.c_int32), ("error", ctypes.c_char * 160)]


class _TuneReport(ctypes.Structure):
    _fields_ = [("trials", ctypes.c_int32), ("improved", ctypes.c_int32), ("base_ms", ctypes.c_double),
                ("best_ms", ctypes.c_double)]


class _EngineStats(ctypes.Structure):
    _fields_ = [("bytes_in_use", ctypes.c_uint64), ("bytes_peak", ctypes.c_uint64), ("plans_cached", ctypes.c_int32),
                ("queued", ctypes.c_int32), ("running", ctypes.c_int32), ("completed", ctypes.c_int64),
                ("plans_built", ctypes.c_int64), ("plans_evicted", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    """The loaded libsnac.so (loaded once). Raises ImportError if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: build it with paper_2106_03583_gb300.build.build()")
        L = ctypes.CDLL(_LIB_PATH)
        vp, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        sig = {
            "snac_plan_create": [ctypes.POINTER(vp), i32, ctypes.POINTER(_Block), i32, ctypes.POINTER(_Options)],
            "snac_plan_workspace_bytes": [vp, ctypes.POINTER(ctypes.c_size_t)],
            "snac_poisson_solve": [vp, vp, vp, f64, vp],
            "snac_plan_info": [vp, ctypes.POINTER(_Info)],
            "snac_plan_mode_cycles": [vp, ctypes.POINTER(i32), i32],
            "snac_plan_destroy": [vp],
            "snac_status_string": [ctypes.c_int],
            "snac_last_error_message": [],
            "snac_apply_operator": [vp, vp, vp, vp],
            "snac_residual": [vp, vp, vp, vp, ctypes.POINTER(f64), vp],
            "snac_residual_ff": [vp, vp, vp, vp, ctypes.POINTER(f64), vp],
            "snac_pencil_forward": [vp, ctypes.c_int64, vp, vp, vp],
            "snac_pencil_backward_update": [vp, ctypes.c_int64, vp, vp, vp],
            "snac_pencil_setup": [vp, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                  ctypes.POINTER(ctypes.c_int64)],
            "snac_pencil_residual": [vp, vp, vp, vp, f64, ctypes.POINTER(f64), vp],
            "snac_mode_solve": [vp, vp, vp, f64, vp],
            "snac_mode_fix_mean": [vp, vp, f64, vp],
            "snac_poisson_solve_batch": [i32, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), f64,
                                         ctypes.POINTER(i32), vp],
            "snac_test_wait_timeout": [vp, f64, vp],
            "snac_forward_transform": [vp, vp, vp, vp],
            "snac_backward_update": [vp, vp, vp, vp],
            "snac_mode_operator": [vp, vp, vp, vp],
            "snac_mode_vcycles": [vp, vp, vp, i32, vp],
            "snac_plan_set_profiling": [vp, i32],
            "snac_plan_kernel_stats": [vp, ctypes.POINTER(_KStat), i32, ctypes.POINTER(i32)],
            "snac_plan_reset_stats": [vp],
            "snac_residual_noalloc": [ctypes.POINTER(_Block), vp, vp, vp, ctypes.POINTER(f64), vp],
            "snac_engine_create": [ctypes.POINTER(vp), ctypes.POINTER(_EngineOptions)],
            "snac_engine_submit": [vp, i32, ctypes.POINTER(_Block), i32, ctypes.POINTER(_Options), vp, vp, f64,
                                   ctypes.POINTER(ctypes.c_int64)],
            "snac_engine_wait": [vp, ctypes.c_int64, ctypes.POINTER(_Info), ctypes.POINTER(_Times)],
            "snac_engine_get_stats": [vp, ctypes.POINTER(_EngineStats)],
            "snac_engine_clock": [],
            "snac_engine_destroy": [vp],
            "snac_autotune": [i32, ctypes.POINTER(_Block), i32, ctypes.POINTER(_Options), vp, f64,
                              ctypes.POINTER(_Options), ctypes.POINTER(_TuneReport), vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name in ("snac_status_string", "snac_last_error_message") else \
                ctypes.c_double if name == "snac_engine_clock" else ctypes.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != SNAC_OK:
        msg = lib().snac_last_error_message()
        raise SnacError(status, msg.decode() if msg else "")


def _marshal_blocks(blocks):
    arr = (_Block * len(blocks))()
    keep = []
    for b, blk in enumerate(blocks):
        c = arr[b]
        for a in range(3):
            c.lo[a] = int(blk["lo"][a])
            c.hi[a] = int(blk["hi"][a])
            w = np.ascontiguousarray(blk["dx"][a], dtype=np.float64)
            keep.append(w)
            c.h_dx[a] = w.ctypes.data
            for s in range(2):
                c.bc[a][s] = _BC[blk["bc"][a][s]]
                c.nbr[a][s] = int(blk["nbr"][a][s])
    return arr, keep


def residual_noalloc(block, rhs, p, r):
    """r = rhs - A p for one block without a plan and without any device allocation
    (``snac_residual_noalloc``), for callers whose device memory is owned by their own allocator or
    budget. rhs, p, r: contiguous CUDA float64 tensors [z][y][x]. Returns (||r||^2, ||rhs||^2)."""
    import torch
    arr, keep = _marshal_blocks([block])
    n = int(np.prod([block["hi"][a] - block["lo"][a] + 1 for a in range(3)]))
    for name, t in (("rhs", rhs), ("p", p), ("r", r)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or \
                not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor with {n} elements")
    norms = (ctypes.c_double * 2)()
    stream = ctypes.c_void_p(torch.cuda.current_stream(rhs.device).cuda_stream)
    _check(lib().snac_residual_noalloc(arr, ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                       ctypes.c_void_p(r.data_ptr()), norms, stream))
    del keep
    return norms[0], norms[1]


class Plan:
    """A solver plan for one multi-block problem (``snac_plan_create``)."""

    def __init__(self, blocks, homog_axis: int = 2, precision: str = "fp64", nu1: int = 2, nu2: int = 2,
                 max_outer: int = 20, max_cycles: int = 40, max_coarse: int = 64, inner_reduction: float = 0.0,
                 fused: int = -1, shift: float = 0.0, modes=None, onchip: bool = True, bottom_cells: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("snac.Plan needs a CUDA device")
        if precision not in _PREC:
            raise ValueError(f"precision must be one of {list(_PREC)}")
        torch.cuda.init()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.blocks = blocks
        self.precision = precision
        self.inner_dtype = torch.float64 if precision == "fp64" else torch.float32
        arr, keep = _marshal_blocks(blocks)
        q0, q1 = modes if modes is not None else (0, 0)
        opt = _Options(_PREC[precision], nu1, nu2, max_outer, max_cycles, max_coarse, fused, inner_reduction, shift,
                       int(q0), int(q1), 0 if onchip else -1, int(bottom_cells))
        h = ctypes.c_void_p()
        _check(lib().snac_plan_create(ctypes.byref(h), len(blocks), arr, homog_axis, ctypes.byref(opt)))
        del keep
        self._h = h
        self.nz = int(blocks[0]["hi"][2] - blocks[0]["lo"][2] + 1)
        self.ncell = int(sum((b["hi"][0] - b["lo"][0] + 1) * (b["hi"][1] - b["lo"][1] + 1) for b in blocks))
        self.n3 = self.ncell * self.nz
        # wavenumbers held in mode space (all, or the range of a wavenumber-range plan)
        self.mode_range = (int(q0), int(q1)) if modes is not None else (0, self.nz)
        self.nmodes = self.mode_range[1] - self.mode_range[0]

    # ---- helpers
    def _stream(self):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _ptr(self, t, dtype, n, name):
        import torch
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch.Tensor")
        if t.device != self.device or t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name} must be a contiguous {dtype} tensor on {self.device} with {n} elements")
        return ctypes.c_void_p(t.data_ptr())

    # ---- the solve
    def solve(self, rhs, p, tol: float = 1e-10, raise_on_error: bool = True) -> dict:
        """Solve A p = rhs in place on p (initial guess in, solution out). Returns info()."""
        import torch
        st = lib().snac_poisson_solve(self._h, self._ptr(rhs, torch.float64, self.n3, "rhs"),
                                      self._ptr(p, torch.float64, self.n3, "p"), float(tol), self._stream())
        if st != SNAC_OK and raise_on_error:
            _check(st)
        return self.info()

    def test_wait_timeout(self, wait_seconds: float = 0.05) -> str:
        """Run the bounded-wait self-test (snac_test_wait_timeout); returns the status name."""
        return STATUS.get(lib().snac_test_wait_timeout(self._h, float(wait_seconds), self._stream()), "?")

    def info(self) -> dict:
        inf = _Info()
        _check(lib().snac_plan_info(self._h, ctypes.byref(inf)))
        d = {k: getattr(inf, k) for k, _ in _Info._fields_}
        d["status_name"] = STATUS.get(d["status"], str(d["status"]))
        return d

    def mode_cycles(self) -> np.ndarray:
        out = (ctypes.c_int32 * self.nmodes)()
        _check(lib().snac_plan_mode_cycles(self._h, out, self.nmodes))
        return np.frombuffer(out, dtype=np.int32).copy()

    # ---- tracing
    def set_profiling(self, enable: bool):
        """CUDA-event timing of every kernel launch of this plan (launch counts are always kept)."""
        _check(lib().snac_plan_set_profiling(self._h, 1 if enable else 0))

    def reset_stats(self):
        _check(lib().snac_plan_reset_stats(self._h))

    def kernel_stats(self) -> dict:
        """{kernel: {launches, ms, bytes, flops}}: bytes/flops are algorithmic, ms needs profiling."""
        n = ctypes.c_int32()
        buf = (_KStat * 32)()
        _check(lib().snac_plan_kernel_stats(self._h, buf, 32, ctypes.byref(n)))
        return {buf[k].name.decode(): {"launches": buf[k].launches, "ms": buf[k].ms, "bytes": buf[k].bytes,
                                       "flops": buf[k].flops} for k in range(n.value)}

    @property
    def workspace_bytes(self) -> int:
        v = ctypes.c_size_t()
        _check(lib().snac_plan_workspace_bytes(self._h, ctypes.byref(v)))
        return int(v.value)

    # ---- stages
    def apply_operator(self, p, out):
        import torch
        _check(lib().snac_apply_operator(self._h, self._ptr(p, torch.float64, self.n3, "p"),
                                         self._ptr(out, torch.float64, self.n3, "out"), self._stream()))

    def residual(self, rhs, p, r):
        import torch
        norms = (ctypes.c_double * 2)()
        _check(lib().snac_residual(self._h, self._ptr(rhs, torch.float64, self.n3, "rhs"),
                                   self._ptr(p, torch.float64, self.n3, "p"),
                                   self._ptr(r, torch.float64, self.n3, "r"), norms, self._stream()))
        return norms[0], norms[1]

    def residual_ff(self, rhs, p, r):
        """r (float32) = rhs - A p in float-float arithmetic (the mixed plans' intermediate pass);
        returns (||r||^2, ||rhs||^2)."""
        import torch
        norms = (ctypes.c_double * 2)()
        _check(lib().snac_residual_ff(self._h, self._ptr(rhs, torch.float64, self.n3, "rhs"),
                                      self._ptr(p, torch.float64, self.n3, "p"),
                                      self._ptr(r, torch.float32, self.n3, "r"), norms, self._stream()))
        return norms[0], norms[1]

    # ---- one rank of a wavenumber-sharded solve (pencils [z][c], slabs [local q][plane cell])
    def pencil_forward(self, x, modes):
        import torch
        nc = x.numel() // self.nz
        _check(lib().snac_pencil_forward(self._h, nc, self._ptr(x, torch.float64, nc * self.nz, "x"),
                                         self._ptr(modes, self.inner_dtype, nc * self.nz, "modes"), self._stream()))

    def pencil_backward_update(self, modes, p):
        import torch
        nc = p.numel() // self.nz
        _check(lib().snac_pencil_backward_update(self._h, nc, self._ptr(modes, self.inner_dtype, nc * self.nz, "modes"),
                                                 self._ptr(p, torch.float64, nc * self.nz, "p"), self._stream()))

    def pencil_setup(self, c0: int, ncols: int) -> np.ndarray:
        """Set this plan's pencil (plane cells c0 .. c0 + ncols - 1); returns its halo cells."""
        cap = 4 * int(ncols) + 8
        buf = (ctypes.c_int64 * cap)()
        n = ctypes.c_int64()
        _check(lib().snac_pencil_setup(self._h, int(c0), int(ncols), buf, cap, ctypes.byref(n)))
        self._pencil = (int(c0), int(ncols), int(n.value))
        return np.frombuffer(buf, dtype=np.int64, count=n.value).copy()

    def pencil_residual(self, f, p_ext, r, fshift: float = 0.0):
        """r = (f - fshift) - A p on the pencil; returns (||r||^2, ||f - fshift||^2, sum V p,
        sum V (f - fshift), sum V |f - fshift|) of the pencil."""
        import torch
        _, nc, nh = self._pencil
        sums = (ctypes.c_double * 5)()
        _check(lib().snac_pencil_residual(self._h, self._ptr(f, torch.float64, nc * self.nz, "f"),
                                          self._ptr(p_ext, torch.float64, (nc + nh) * self.nz, "p_ext"),
                                          self._ptr(r, torch.float64, nc * self.nz, "r"), float(fshift), sums,
                                          self._stream()))
        return tuple(sums)

    def mode_solve(self, rhs, sol, target: float) -> dict:
        n = self.nmodes * self.ncell
        _check(lib().snac_mode_solve(self._h, self._ptr(rhs, self.inner_dtype, n, "rhs"),
                                     self._ptr(sol, self.inner_dtype, n, "sol"), float(target), self._stream()))
        return self.info()

    def mode_fix_mean(self, sol, sum_vp: float):
        _check(lib().snac_mode_fix_mean(self._h, self._ptr(sol, self.inner_dtype, self.nmodes * self.ncell, "sol"),
                                        float(sum_vp), self._stream()))

    def forward_transform(self, x, modes):
        import torch
        _check(lib().snac_forward_transform(self._h, self._ptr(x, torch.float64, self.n3, "x"),
                                            self._ptr(modes, self.inner_dtype, self.n3, "modes"), self._stream()))

    def backward_update(self, modes, p):
        import torch
        _check(lib().snac_backward_update(self._h, self._ptr(modes, self.inner_dtype, self.n3, "modes"),
                                          self._ptr(p, torch.float64, self.n3, "p"), self._stream()))

    def mode_operator(self, u, out):
        n = self.nmodes * self.ncell
        _check(lib().snac_mode_operator(self._h, self._ptr(u, self.inner_dtype, n, "u"),
                                        self._ptr(out, self.inner_dtype, n, "out"), self._stream()))

    def mode_vcycles(self, f, u, ncycles: int = 1):
        n = self.nmodes * self.ncell
        _check(lib().snac_mode_vcycles(self._h, self._ptr(f, self.inner_dtype, n, "f"),
                                       self._ptr(u, self.inner_dtype, n, "u"), int(ncycles), self._stream()))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().snac_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve_batch(plans, rhs, p, tol: float = 1e-10, raise_on_error: bool = True) -> list:
    """Solve several problems together (snac_poisson_solve_batch): plans[k] with rhs[k] -> p[k]
    (CUDA float64 tensors as in Plan.solve). Returns each plan's info()."""
    import torch
    n = len(plans)
    if not (len(rhs) == len(p) == n) or n == 0:
        raise ValueError("one rhs and one p per plan")
    hs = (ctypes.c_void_p * n)(*[pl._h.value for pl in plans])
    fs = (ctypes.c_void_p * n)(*[pl._ptr(r, torch.float64, pl.n3, "rhs").value for pl, r in zip(plans, rhs)])
    ps = (ctypes.c_void_p * n)(*[pl._ptr(x, torch.float64, pl.n3, "p").value for pl, x in zip(plans, p)])
    st = (ctypes.c_int32 * n)()
    rc = lib().snac_poisson_solve_batch(n, hs, fs, ps, float(tol), st, plans[0]._stream())
    if rc != SNAC_OK and raise_on_error:
        _check(rc)
    return [pl.info() for pl in plans]


class Engine:
    """Serving engine (``include/snac_engine.h``): solves of different problems submitted at any time,
    admitted under a device-memory budget, run concurrently by ``workers`` threads / CUDA streams
    with resident cached plans; requests of small (on-chip) problems that are ready together are
    solved in one batched solve of up to ``max_group``. Host arrays in, host arrays out.

        eng = snac.Engine(workers=4, hbm_budget=150e9)
        t = eng.submit(blocks, f, tol=1e-10, precision="mixed")
        p, info, times = eng.wait(t)
    """

    def __init__(self, workers: int = 4, hbm_budget: float = 150e9, max_cached_plans: int = 64,
                 autotune: bool = False, max_group: int = 16):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("snac.Engine needs a CUDA device")
        torch.cuda.init()
        opt = _EngineOptions(int(workers), int(max_cached_plans), int(hbm_budget), 1 if autotune else 0,
                             int(max_group))
        h = ctypes.c_void_p()
        _check(lib().snac_engine_create(ctypes.byref(h), ctypes.byref(opt)))
        self._h = h
        self._live = {}   # ticket -> (rhs, p) kept alive until wait

    def submit(self, blocks, rhs, tol: float = 1e-10, precision: str = "fp64", homog_axis: int = 2, nu1: int = 2,
               nu2: int = 2, max_outer: int = 20, max_cycles: int = 40, max_coarse: int = 64,
               inner_reduction: float = 0.0, fused: int = -1, shift: float = 0.0, onchip: bool = True,
               bottom_cells: int = 0) -> int:
        if precision not in _PREC:
            raise ValueError(f"precision must be one of {list(_PREC)}")
        n3 = int(sum(np.prod([b["hi"][a] - b["lo"][a] + 1 for a in range(3)]) for b in blocks))
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        if rhs.shape != (n3,):
            raise ValueError(f"rhs must be a float64 array of {n3} elements")
        p = np.empty(n3, dtype=np.float64)
        arr, keep = _marshal_blocks(blocks)
        opt = _Options(_PREC[precision], nu1, nu2, max_outer, max_cycles, max_coarse, fused, inner_reduction, shift,
                       onchip=0 if onchip else -1, bottom_cells=int(bottom_cells))
        t = ctypes.c_int64()
        _check(lib().snac_engine_submit(self._h, len(blocks), arr, homog_axis, ctypes.byref(opt),
                                        ctypes.c_void_p(rhs.ctypes.data), ctypes.c_void_p(p.ctypes.data),
                                        float(tol), ctypes.byref(t)))
        del keep   # the engine copied the block descriptions
        self._live[t.value] = (rhs, p)
        return t.value

    def wait(self, ticket: int, raise_on_error: bool = True):
        """(solution, info dict, times dict) of a request; blocks until it is complete."""
        inf, tm = _Info(), _Times()
        st = lib().snac_engine_wait(self._h, int(ticket), ctypes.byref(inf), ctypes.byref(tm))
        rhs, p = self._live.pop(ticket, (None, None))
        if st != SNAC_OK and raise_on_error:
            _check(st)
        info = {k: getattr(inf, k) for k, _ in _Info._fields_}
        info["status"] = st
        info["status_name"] = STATUS.get(st, str(st))
        times = {k: getattr(tm, k) for k, _ in _Times._fields_}
        times["error"] = tm.error.decode(errors="replace")
        return p, info, times

    def stats(self) -> dict:
        s = _EngineStats()
        _check(lib().snac_engine_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _EngineStats._fields_}

    @staticmethod
    def clock() -> float:
        return float(lib().snac_engine_clock())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().snac_engine_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


_OPTION_NAMES = ("nu1", "nu2", "max_outer", "max_cycles", "max_coarse", "fused", "inner_reduction", "shift")
_TUNED_EXTRA = ("bottom_cells",)


def autotune(blocks, rhs, tol: float = 1e-10, precision: str = "fp64", homog_axis: int = 2, **base):
    """``snac_autotune``: the fastest multigrid schedule for this problem, found by timing complete
    solves of ``rhs`` (a CUDA float64 tensor in the caller layout) on the current stream.
    ``base`` overrides the starting options (Plan's keywords). Returns (options for Plan, report)."""
    import torch
    if precision not in _PREC:
        raise ValueError(f"precision must be one of {list(_PREC)}")
    n3 = int(sum(np.prod([b["hi"][a] - b["lo"][a] + 1 for a in range(3)]) for b in blocks))
    if not isinstance(rhs, torch.Tensor) or not rhs.is_cuda or rhs.dtype != torch.float64 or \
            not rhs.is_contiguous() or rhs.numel() != n3:
        raise ValueError(f"rhs must be a contiguous CUDA float64 tensor with {n3} elements")
    d = dict(nu1=2, nu2=2, max_outer=20, max_cycles=40, max_coarse=64, fused=-1, inner_reduction=0.0, shift=0.0,
             bottom_cells=0)
    unknown = set(base) - set(d)
    if unknown:
        raise ValueError(f"unknown options {sorted(unknown)}")
    d.update(base)
    opt = _Options(_PREC[precision], *(d[k] for k in _OPTION_NAMES), bottom_cells=int(d["bottom_cells"]))
    best, rep = _Options(), _TuneReport()
    arr, keep = _marshal_blocks(blocks)
    stream = ctypes.c_void_p(torch.cuda.current_stream(rhs.device).cuda_stream)
    _check(lib().snac_autotune(len(blocks), arr, homog_axis, ctypes.byref(opt), ctypes.c_void_p(rhs.data_ptr()),
                               float(tol), ctypes.byref(best), ctypes.byref(rep), stream))
    del keep
    chosen = {k: getattr(best, k) for k in _OPTION_NAMES + _TUNED_EXTRA}
    chosen["onchip"] = best.onchip == 0
    chosen["precision"] = precision
    return chosen, {k: getattr(rep, k) for k, _ in _TuneReport._fields_}
