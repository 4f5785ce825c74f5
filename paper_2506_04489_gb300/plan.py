"""Python face of the C ABI: a solver plan bound to torch tensors and streams."""
from __future__ import annotations

import ctypes

import numpy as np

_PREC = {"fp64": 0, "fp32": 1, "mixed": 2, "df32": 3}


def precision_dtype(precision: str):
    import torch
    return torch.float32 if precision == "fp32" else torch.float64


def _vec3(v):
    if np.isscalar(v):
        return (v, v, v)
    v = tuple(v)
    if len(v) != 3:
        raise ValueError("expected a scalar or 3 values")
    return v


def torch_empty_pinned(shape, dtype):
    import torch
    return torch.empty(shape, dtype=dtype, pin_memory=True)


def torch_allocator():
    """An sp_allocator drawing on PyTorch's CUDA caching allocator (argument marshalling
    only: the callbacks hand torch's blocks to the library and give them back)."""
    from . import _native as N

    def alloc(nbytes, device, ctx):
        import torch
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=int(device)))
        except Exception:
            return None

    def release(ptr, nbytes, device, ctx):
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))

    cb = N.Allocator(N.ALLOC_FN(alloc), N.RELEASE_FN(release), None)
    return cb


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """Solver plan: ``Plan(n, lo, hi, precision="fp64")`` then ``solve(rho)``.

    n, lo, hi : grid points and box faces per axis (scalars apply to all axes).
    precision : "fp64", "fp32", "mixed" (float64 I/O, FP32 passes) or "df32" (float64
                I/O, double-float passes on the FP32 pipes).
    eps       : GS cutoff when the GS table is generated (default 1e-4, Alg. 1).
    gs        : optional explicit GS table (weights, exponents) as float64 arrays.
    max_batch : largest batch for ``solve_batched``.
    precompute: run Alg. 1 on the current stream at construction.
    kernel    : "superpotential" (the paper's method) or "gs_plain" (the original GS
                method without near-field correction, for comparison).
    allocator : None (the library allocates with cudaMalloc) or "torch" (the plan's device
                memory comes from PyTorch's caching allocator, sp_plan_create_ex).
    """

    def __init__(self, n, lo, hi, precision: str = "fp64", eps: float = 1e-4, gs=None,
                 max_batch: int = 1, precompute: bool = True, stream=None, kernel: str = "superpotential",
                 allocator=None):
        from . import _native as N
        self._N = N
        if precision not in _PREC:
            raise ValueError(f"precision must be one of {list(_PREC)}")
        self.n = tuple(int(x) for x in _vec3(n))
        self.lo = tuple(float(x) for x in _vec3(lo))
        self.hi = tuple(float(x) for x in _vec3(hi))
        self.precision = precision
        self.max_batch = int(max_batch)
        n_c = (ctypes.c_int * 3)(*self.n)
        lo_c = (ctypes.c_double * 3)(*self.lo)
        hi_c = (ctypes.c_double * 3)(*self.hi)
        if gs is not None:
            w = np.ascontiguousarray(gs[0], dtype=np.float64)
            a = np.ascontiguousarray(gs[1], dtype=np.float64)
            wp, ap, terms = w.ctypes.data_as(N._dp), a.ctypes.data_as(N._dp), len(w)
        else:
            wp = ap = None
            terms = 0
        h = ctypes.c_void_p()
        if allocator not in (None, "torch"):
            raise ValueError("allocator must be None or 'torch'")
        # the callbacks must outlive the plan: keep them on it
        self._allocator = torch_allocator() if allocator == "torch" else None
        N.check(N.lib.sp_plan_create_ex(ctypes.byref(h), n_c, lo_c, hi_c, 2, wp, ap, terms, float(eps),
                                        _PREC[precision], self.max_batch,
                                        ctypes.byref(self._allocator) if self._allocator else None),
                "sp_plan_create_ex")
        self._h = h
        self.dtype = precision_dtype(precision)
        if kernel not in ("superpotential", "gs_plain"):
            raise ValueError("kernel must be 'superpotential' or 'gs_plain'")
        self.kernel = kernel
        if kernel == "gs_plain":
            N.check(N.lib.sp_plan_set_kernel(h, 1), "sp_plan_set_kernel")
        if precompute:
            self.precompute(stream)

    # ----------------------------------------------------------------- lifecycle
    def precompute(self, stream=None) -> None:
        self._N.check(self._N.lib.sp_kernel_precompute(self._h, _stream_handle(stream)), "sp_kernel_precompute")

    def sync(self) -> None:
        """Wait for the plan's last work and raise on an error its kernels reported
        (sp_plan_sync: SP_ERR_TIMEOUT for a bounded wait that gave up)."""
        self._N.check(self._N.lib.sp_plan_sync(self._h), "sp_plan_sync")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._N.check(self._N.lib.sp_plan_destroy(self._h), "sp_plan_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def workspace_bytes(self) -> int:
        return int(self._N.lib.sp_plan_workspace_bytes(self._h))

    @property
    def gs_terms(self) -> int:
        return int(self._N.lib.sp_plan_gs_terms(self._h))

    # ----------------------------------------------------------------- solves
    def _check_io(self, t, batch: bool):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("expected a CUDA torch.Tensor")
        if t.dtype != self.dtype:
            raise TypeError(f"expected dtype {self.dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        shape = tuple(t.shape[1:]) if batch else tuple(t.shape)
        if shape != self.n:
            raise ValueError(f"expected grid shape {self.n}, got {shape}")

    def solve(self, rho, out=None, stream=None):
        """u = crop(IDFT3(M .* DFT3(pad(rho)))) (Alg. 2); ``out`` may be ``rho``.

        A CPU ``rho`` (pinned for asynchronous copies) is copied to a device staging
        buffer, solved there and copied back into ``out`` (a CPU tensor, allocated
        pinned if not given); the copies are ordered on the same stream.
        """
        import torch
        if isinstance(rho, torch.Tensor) and not rho.is_cuda:
            return self._solve_host(rho, out, stream)
        self._check_io(rho, False)
        if out is None:
            out = torch.empty_like(rho)
        self._check_io(out, False)
        self._N.check(self._N.lib.sp_solve(self._h, ctypes.c_void_p(rho.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), "sp_solve")
        return out

    def _solve_host(self, rho, out, stream):
        if out is None:
            out = torch_empty_pinned(self.n, self.dtype)
        self.solve_host_stream([rho], [out], stream, wait=False)
        return out

    # ----------------------------------------------------------------- batched execution
    def autotune(self, batch: int = 1, stream=None) -> dict:
        """Pick the pass tiles and the line passes' radix plans for `batch` right-hand
        sides by timing; returns launch_config()."""
        self._N.check(self._N.lib.sp_plan_autotune(self._h, int(batch), _stream_handle(stream)), "sp_plan_autotune")
        return self.launch_config()

    def launch_config(self) -> dict:
        """Tiles, radix-plan choice per axis and the radices of the passes in use."""
        line = (ctypes.c_int * 3)()
        z = ctypes.c_int()
        plan = (ctypes.c_int * 3)()
        rad = (ctypes.c_int * 24)()
        sched = ctypes.c_int()
        self._N.check(self._N.lib.sp_plan_launch_config(self._h, line, ctypes.byref(z), plan, rad, ctypes.byref(sched)),
                      "sp_plan_launch_config")
        radices = {ax: tuple(r for r in rad[8 * i:8 * i + 8] if r) for i, ax in enumerate(("x", "y", "z"))}
        schedule = {0: "five_passes", 1: "fused_planes", 2: "persistent"}[sched.value]
        return {"line": tuple(line), "z": z.value, "line_plan": tuple(plan), "radices": radices, "schedule": schedule}

    def set_launch_config(self, line=None, z: int = None, line_plan=None, schedule: str = None) -> None:
        """Set tiles, line radix plans and the schedule ("five_passes" or "fused_planes")
        (sp_plan_set_launch_config); None keeps a part."""
        cur = self.launch_config()
        lt = (ctypes.c_int * 3)(*(line if line is not None else cur["line"]))
        lp = (ctypes.c_int * 3)(*(line_plan if line_plan is not None else cur["line_plan"]))
        sc = {None: -1, "five_passes": 0, "fused_planes": 1}[schedule]
        self._N.check(self._N.lib.sp_plan_set_launch_config(self._h, lt, int(cur["z"] if z is None else z), lp, sc),
                      "sp_plan_set_launch_config")

    def tiles(self) -> dict:
        line = (ctypes.c_int * 3)()
        z = ctypes.c_int()
        self._N.check(self._N.lib.sp_plan_tiles(self._h, line, ctypes.byref(z)), "sp_plan_tiles")
        return {"line": tuple(line), "z": z.value}

    def set_persistent(self, enable: bool = True) -> None:
        """Run solves as one persistent cooperative launch (sp_plan_set_persistent)."""
        self._N.check(self._N.lib.sp_plan_set_persistent(self._h, int(bool(enable))), "sp_plan_set_persistent")

    def barrier_check(self, blocks: int, expected: int, limit_ms: float = 50.0, stream=None) -> None:
        """Diagnostic of the bounded grid wait (sp_plan_barrier_check); see sync()."""
        self._N.check(self._N.lib.sp_plan_barrier_check(self._h, int(blocks), int(expected), float(limit_ms),
                                                        _stream_handle(stream)), "sp_plan_barrier_check")

    def capture(self, rho, out, stream):
        """CUDA graph of solve_batched(rho, out) on these buffers; replay with Graph.launch."""
        self._check_io(rho, True)
        self._check_io(out, True)
        g = ctypes.c_void_p()
        self._N.check(self._N.lib.sp_graph_capture(self._h, ctypes.c_void_p(rho.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr()), int(rho.shape[0]),
                                                   ctypes.c_void_p(stream.cuda_stream), ctypes.byref(g)),
                      "sp_graph_capture")
        return Graph(self, g, (rho, out))

    def solve_host_stream(self, inputs, outputs, stream=None, wait: bool = True):
        """Solve a sequence of CPU densities into CPU outputs (contiguous tensors of the
        plan's shape and dtype, pinned for overlap) through sp_solve_host: the copy of
        input i+1 and of result i-1 overlap the solve of i.  With ``wait`` (default) it
        returns after the last result is on the host; else the results are complete when
        the work on ``stream`` is."""
        import torch
        if len(inputs) != len(outputs):
            raise ValueError("inputs and outputs must have the same length")
        for t in list(inputs) + list(outputs):
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != self.dtype or tuple(t.shape) != self.n \
                    or not t.is_contiguous():
                raise ValueError(f"expected contiguous CPU {self.dtype} tensors of shape {self.n}")
        n = len(inputs)
        rin = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in inputs])
        rout = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in outputs])
        st = stream if stream is not None else torch.cuda.current_stream()
        self._N.check(self._N.lib.sp_solve_host(self._h, rin, rout, n, ctypes.c_void_p(st.cuda_stream)),
                      "sp_solve_host")
        if wait:
            st.synchronize()
        return outputs

    # ----------------------------------------------------------------- diagnostics
    def set_timing(self, enable, reserve: int = 1) -> None:
        """Turn pass timing on (events for `reserve` solves created now) or off."""
        n = max(1, int(reserve)) if enable else 0
        self._N.check(self._N.lib.sp_plan_set_timing(self._h, n), "sp_plan_set_timing")

    def pass_times(self):
        """{pass name: (total ms, launches)} over the solves recorded since the last call."""
        N = self._N
        tot = (ctypes.c_double * 16)()
        cnt = (ctypes.c_int * 16)()
        names = (ctypes.c_char_p * 16)()
        np_ = N.lib.sp_plan_pass_times(self._h, tot, cnt, names, 16)
        if np_ < 0:
            raise N.SuperpotError(1, "sp_plan_pass_times")
        return {names[i].decode(): (tot[i], cnt[i]) for i in range(np_)}

    def solve_batched(self, rho, out=None, stream=None):
        import torch
        self._check_io(rho, True)
        if out is None:
            out = torch.empty_like(rho)
        self._check_io(out, True)
        self._N.check(self._N.lib.sp_solve_batched(self._h, ctypes.c_void_p(rho.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr()), int(rho.shape[0]),
                                                   _stream_handle(stream)), "sp_solve_batched")
        return out

    def forward_spectrum(self, rho, stream=None):
        """Diagnostic: padded forward DFT, [2n0, 2n1, n2+1] complex (pass precision)."""
        import torch
        self._check_io(rho, False)
        shape = (2 * self.n[0], 2 * self.n[1], self.n[2] + 1)
        if self.precision == "df32":  # (re.hi, im.hi, re.lo, im.lo) float32 per value
            spec = torch.empty(shape + (4,), dtype=torch.float32, device=rho.device)
        else:
            cdt = torch.complex128 if self.precision == "fp64" else torch.complex64
            spec = torch.empty(shape, dtype=cdt, device=rho.device)
        self._N.check(self._N.lib.sp_forward_spectrum(self._h, ctypes.c_void_p(rho.data_ptr()),
                                                      ctypes.c_void_p(spec.data_ptr()), _stream_handle(stream)),
                      "sp_forward_spectrum")
        return spec

    def tables(self, axis: int = 0):
        """Host copies of the FP64 setup tables (synchronises the device)."""
        N = self._N
        S = self.gs_terms
        w = np.empty(S)
        a = np.empty(S)
        M = np.empty(tuple(m + 1 for m in self.n))
        G = np.empty((S, self.n[axis] + 1))
        H = np.empty((S, self.n[axis] + 1))
        d = lambda x: x.ctypes.data_as(N._dp)
        N.check(N.lib.sp_plan_copy_tables(self._h, d(w), d(a), d(M), int(axis), d(G), d(H)), "sp_plan_copy_tables")
        return {"gs_w": w, "gs_a": a, "M": M, "G": G, "H": H}


class Graph:
    """A captured batched solve (holds references to its plan and buffers)."""

    def __init__(self, plan, handle, buffers):
        self._plan = plan
        self._h = handle
        self._buffers = buffers

    def launch(self, stream=None) -> None:
        N = self._plan._N
        N.check(N.lib.sp_graph_launch(self._h, _stream_handle(stream)), "sp_graph_launch")

    def close(self) -> None:
        if self._h is not None and self._h.value:
            N = self._plan._N
            N.check(N.lib.sp_graph_destroy(self._h), "sp_graph_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
