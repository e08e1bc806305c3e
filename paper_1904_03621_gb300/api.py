"""PyTorch-facing API: device memory, streams and argument marshalling only.

Every step of the search runs in libbf's CUDA kernels; this module
allocates the workspace and outputs with torch and passes raw pointers.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

_DTYPES = {torch.int32: _lib.BF_I32, torch.float32: _lib.BF_F32, torch.float64: _lib.BF_F64}


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _options(variant=0, fixed_bits=0, fixed_value=0, task_log2=0, grid_blocks=0, spill_log2=0, profile=0,
             stall_test=0, inner_bits=0):
    return _lib.Options(variant=variant, fixed_bits=fixed_bits, fixed_value=fixed_value,
                        task_log2=task_log2, grid_blocks=grid_blocks, spill_log2=spill_log2, profile=profile,
                        stall_test=stall_test, inner_bits=inner_bits)


def workspace_size(n: int, S: int, dtype: torch.dtype, **opts) -> int:
    lib = _lib.load()
    o = _options(**opts)
    nbytes = lib.bf_workspace_size(n, S, _DTYPES[dtype], ctypes.byref(o))
    if nbytes == 0:
        raise _lib.BFError(_lib.BF_EINVAL, lib.bf_last_error_detail().decode())
    return int(nbytes)


def low_spectrum(J: torch.Tensor, h: torch.Tensor, S: int, *, variant: int = 0, fixed_bits: int = 0,
                 fixed_value: int = 0, task_log2: int = 0, grid_blocks: int = 0, spill_log2: int = 0,
                 profile: int = 0, stream=None, workspace: torch.Tensor | None = None, check: bool = True,
                 out: tuple | None = None, stall_test: int = 0, inner_bits: int = 0):
    """S lowest (energy, configuration) pairs of E(s) = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i.

    J: (n, n) CUDA tensor (int32, float32 or float64), strict upper triangle read.
    h: (n,) CUDA tensor of the same dtype.
    Returns (energies, states): energies int64 (int32 input) or float64, states as
    int64 tensors holding the uint64 configuration integers (bit i = spin i is +1).
    With check=True the stream is synchronised and device-side errors raise.
    """
    lib = _lib.load()
    if J.dtype not in _DTYPES or h.dtype != J.dtype:
        raise TypeError("J and h must share one of int32, float32, float64")
    if not (J.is_cuda and h.is_cuda):
        raise ValueError("J and h must be CUDA tensors")
    n = J.shape[0]
    J = J.contiguous()
    h = h.contiguous()
    o = _options(variant, fixed_bits, fixed_value, task_log2, grid_blocks, spill_log2, profile, stall_test,
                 inner_bits)
    nbytes = lib.bf_workspace_size(n, S, _DTYPES[J.dtype], ctypes.byref(o))
    if nbytes == 0:
        # the call validates its arguments before touching any pointer: get the exact status
        _lib.check(lib.bf_low_spectrum(None, None, n, S, _DTYPES[J.dtype], None, None, None, 0,
                                       ctypes.byref(o), None), lib)
        raise _lib.BFError(_lib.BF_EINVAL, lib.bf_last_error_detail().decode())
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=J.device)
    edt = torch.int64 if J.dtype == torch.int32 else torch.float64
    if out is not None:
        energies, states = out
    else:
        energies = torch.empty(S, dtype=edt, device=J.device)
        states = torch.empty(S, dtype=torch.int64, device=J.device)
    sh = _stream_handle(stream)
    st = lib.bf_low_spectrum(J.data_ptr(), h.data_ptr(), n, S, _DTYPES[J.dtype], energies.data_ptr(),
                             states.data_ptr(), workspace.data_ptr(), workspace.numel(), ctypes.byref(o), sh)
    _lib.check(st, lib)
    if check:
        _lib.check(lib.bf_workspace_status(workspace.data_ptr(), sh), lib)
    return energies, states


def autotune(J: torch.Tensor, h: torch.Tensor, S: int, *, fixed_bits: int = 0, fixed_value: int = 0,
             spill_log2: int = 0, stream=None) -> dict:
    """Time the candidate kernels and launch shapes of low_spectrum for this search size (bf_autotune).

    Returns {"variant", "inner_bits", "task_log2", "grid_blocks", "configs_per_s", "candidates"}
    (every candidate with its measured rate); the choice is cached in the library for this device
    and (n, n - fixed_bits, S, dtype), so later calls that leave variant, inner_bits, task_log2 and
    grid_blocks at 0 use it.
    """
    lib = _lib.load()
    if J.dtype not in _DTYPES or h.dtype != J.dtype:
        raise TypeError("J and h must share one of int32, float32, float64")
    n = J.shape[0]
    J = J.contiguous()
    h = h.contiguous()
    base = _options(0, fixed_bits, fixed_value, 0, 0, spill_log2)
    nbytes = lib.bf_workspace_size(n, S, _DTYPES[J.dtype], ctypes.byref(_options(1, fixed_bits, fixed_value, 0, 0,
                                                                                   spill_log2)))
    if nbytes == 0:
        raise _lib.BFError(_lib.BF_EINVAL, lib.bf_last_error_detail().decode())
    ws = torch.empty(nbytes, dtype=torch.uint8, device=J.device)
    edt = torch.int64 if J.dtype == torch.int32 else torch.float64
    en = torch.empty(S, dtype=edt, device=J.device)
    st = torch.empty(S, dtype=torch.int64, device=J.device)
    best = _lib.Options()
    rate = ctypes.c_double(0.0)
    recs = (_lib.TuneRecord * 64)()
    count = ctypes.c_int(0)
    _lib.check(lib.bf_autotune(J.data_ptr(), h.data_ptr(), n, S, _DTYPES[J.dtype], en.data_ptr(), st.data_ptr(),
                               ws.data_ptr(), nbytes, ctypes.byref(base), _stream_handle(stream), ctypes.byref(best),
                               ctypes.byref(rate), recs, 64, ctypes.byref(count)), lib)

    def brief(o):
        return {"variant": o.variant, "inner_bits": o.inner_bits, "task_log2": o.task_log2,
                "grid_blocks": o.grid_blocks}

    out = brief(best)
    out["configs_per_s"] = float(rate.value)
    out["candidates"] = [dict(brief(recs[i].opt), configs_per_s=float(recs[i].configs_per_s))
                         for i in range(count.value)]
    return out


def low_spectrum_qubo(a: torch.Tensor, b: torch.Tensor, S: int, *, variant: int = 0, fixed_bits: int = 0,
                      fixed_value: int = 0, task_log2: int = 0, grid_blocks: int = 0, spill_log2: int = 0,
                      stream=None, workspace: torch.Tensor | None = None, check: bool = True):
    """S lowest (F, configuration) pairs of the QUBO form (Sec. 2, Eqs. (2)-(3)).

    F(q) = sum_{i<j} a_ij q_i q_j + sum_i b_i q_i over q in {0,1}^n (the paper's Eq. (2)
    with the overall sign flipped, as for Eq. (1)); configuration bit i = q_i.
    a: (n, n) CUDA tensor (int32, float32 or float64), strict upper triangle read; b: (n,).
    Returns (F, states): F int64 (exact, int32 input) or float64.
    """
    lib = _lib.load()
    if a.dtype not in _DTYPES or b.dtype != a.dtype:
        raise TypeError("a and b must share one of int32, float32, float64")
    if not (a.is_cuda and b.is_cuda):
        raise ValueError("a and b must be CUDA tensors")
    n = a.shape[0]
    a = a.contiguous()
    b = b.contiguous()
    o = _options(variant, fixed_bits, fixed_value, task_log2, grid_blocks, spill_log2, 0)
    nbytes = lib.bf_qubo_workspace_size(n, S, _DTYPES[a.dtype], ctypes.byref(o))
    if nbytes == 0:
        _lib.check(lib.bf_low_spectrum_qubo(None, None, n, S, _DTYPES[a.dtype], None, None, None, 0,
                                            ctypes.byref(o), None), lib)
        raise _lib.BFError(_lib.BF_EINVAL, lib.bf_last_error_detail().decode())
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=a.device)
    edt = torch.int64 if a.dtype == torch.int32 else torch.float64
    F = torch.empty(S, dtype=edt, device=a.device)
    states = torch.empty(S, dtype=torch.int64, device=a.device)
    sh = _stream_handle(stream)
    st = lib.bf_low_spectrum_qubo(a.data_ptr(), b.data_ptr(), n, S, _DTYPES[a.dtype], F.data_ptr(),
                                  states.data_ptr(), workspace.data_ptr(), workspace.numel(), ctypes.byref(o), sh)
    _lib.check(st, lib)
    if check:
        _lib.check(lib.bf_workspace_status(workspace.data_ptr(), sh), lib)
    return F, states


def low_spectrum_potts(J: torch.Tensor, h: torch.Tensor, S: int, *, task_log2: int = 0, grid_blocks: int = 0,
                       spill_log2: int = 0, profile: int = 0, stream=None, workspace: torch.Tensor | None = None,
                       check: bool = True, out: tuple | None = None):
    """S lowest (energy, configuration) pairs of the q-state Potts model.

    E(sigma) = sum_{i<j} J_ij [sigma_i == sigma_j] + sum_i h_i(sigma_i), sigma_i in {0..q-1};
    configuration c = sum_i sigma_i q^i.  J: (n, n) CUDA tensor, strict upper triangle read;
    h: (n, q) CUDA tensor of the same dtype (q = h.shape[1], 2..8).  Returns (energies, states).
    """
    lib = _lib.load()
    if J.dtype not in _DTYPES or h.dtype != J.dtype:
        raise TypeError("J and h must share one of int32, float32, float64")
    if not (J.is_cuda and h.is_cuda):
        raise ValueError("J and h must be CUDA tensors")
    if h.dim() != 2 or h.shape[0] != J.shape[0]:
        raise ValueError("h must have shape (n, q)")
    n, q = J.shape[0], h.shape[1]
    J = J.contiguous()
    h = h.contiguous()
    o = _options(0, 0, 0, task_log2, grid_blocks, spill_log2, profile)
    nbytes = lib.bf_potts_workspace_size(n, q, S, _DTYPES[J.dtype], ctypes.byref(o))
    if nbytes == 0:
        _lib.check(lib.bf_low_spectrum_potts(None, None, n, q, S, _DTYPES[J.dtype], None, None, None, 0,
                                             ctypes.byref(o), None), lib)
        raise _lib.BFError(_lib.BF_EINVAL, lib.bf_last_error_detail().decode())
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=J.device)
    edt = torch.int64 if J.dtype == torch.int32 else torch.float64
    if out is not None:
        energies, states = out
    else:
        energies = torch.empty(S, dtype=edt, device=J.device)
        states = torch.empty(S, dtype=torch.int64, device=J.device)
    sh = _stream_handle(stream)
    st = lib.bf_low_spectrum_potts(J.data_ptr(), h.data_ptr(), n, q, S, _DTYPES[J.dtype], energies.data_ptr(),
                                   states.data_ptr(), workspace.data_ptr(), workspace.numel(), ctypes.byref(o), sh)
    _lib.check(st, lib)
    if check:
        _lib.check(lib.bf_workspace_status(workspace.data_ptr(), sh), lib)
    return energies, states


def states_u64(states: torch.Tensor) -> np.ndarray:
    """Configuration integers as numpy uint64 (the int64 tensor holds their bits)."""
    return states.detach().cpu().numpy().view(np.uint64)


def last_profile_ms() -> float:
    """Enumeration-kernel time (ms) of the last call made with profile=1 on this thread."""
    lib = _lib.load()
    ms = ctypes.c_float(0.0)
    _lib.check(lib.bf_last_profile(ctypes.byref(ms)), lib)
    return float(ms.value)


def issue_rates(stream=None) -> dict:
    """Measured issue rates of the current GPU (bf_measure_issue_rates): lane-instructions per
    clock per SM of 3-input integer adds, 3-input logic operations, 16x2 min/max and FP32 FMA,
    the SM count and the SM clock seen by the probe."""
    lib = _lib.load()
    ws = torch.empty(int(lib.bf_issue_rates_workspace_size()), dtype=torch.uint8, device="cuda")
    r = _lib.IssueRates()
    _lib.check(lib.bf_measure_issue_rates(ws.data_ptr(), ws.numel(), ctypes.byref(r), _stream_handle(stream)), lib)
    return {k: getattr(r, k) for k, _ in _lib.IssueRates._fields_}


def launch_count() -> int:
    """Kernels launched by libbf in this process so far."""
    return int(_lib.load().bf_launch_count())


_NP = {torch.int32: np.int32, torch.float32: np.float32, torch.float64: np.float64}


def pack_batch(instance_list, dtype: torch.dtype = torch.float64, device="cuda"):
    """Pack [(J, h, ...), ...] into the device arrays bf_low_spectrum_batched takes.

    Returns (J_packed, J_offsets, h_packed, h_offsets, n, n_max); integer couplings are
    carried exactly when dtype is float64.
    """
    from . import instances as inst
    n, Jp, Jo, hp, ho = inst.pack(instance_list, dtype=_NP[dtype])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
    return t(Jp), t(Jo), t(hp), t(ho), t(n), int(n.max())


def batched_workspace_size(B: int, n_max: int, S: int, dtype: torch.dtype, **opts) -> int:
    lib = _lib.load()
    o = _options(**opts)
    nbytes = lib.bf_batched_workspace_size(B, n_max, S, _DTYPES[dtype], ctypes.byref(o))
    if nbytes == 0:
        raise _lib.BFError(_lib.BF_EINVAL, lib.bf_last_error_detail().decode())
    return int(nbytes)


def low_spectrum_batched(J_packed, J_offsets, h_packed, h_offsets, n, S: int, *, n_max: int,
                         task_log2: int = 0, grid_blocks: int = 0, stream=None,
                         workspace: torch.Tensor | None = None, check: bool = True, out: tuple | None = None):
    """S lowest (energy, configuration) pairs of each of B instances in one launch sequence.

    All tensors live on the same CUDA device: J_packed / h_packed (int32, float32 or
    float64), J_offsets / h_offsets (int64 element offsets), n (int32 spin counts).
    Returns (energies (B, S), states (B, S)).  With check=False nothing synchronises,
    so the call can be captured in a CUDA graph (pass workspace and out then).
    """
    lib = _lib.load()
    dt = J_packed.dtype
    if dt not in _DTYPES or h_packed.dtype != dt:
        raise TypeError("J_packed and h_packed must share one of int32, float32, float64")
    B = n.shape[0]
    o = _options(0, 0, 0, task_log2, grid_blocks)
    nbytes = lib.bf_batched_workspace_size(B, n_max, S, _DTYPES[dt], ctypes.byref(o))
    if nbytes == 0:
        raise _lib.BFError(_lib.BF_EINVAL, lib.bf_last_error_detail().decode())
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=J_packed.device)
    if out is not None:
        energies, states = out
    else:
        edt = torch.int64 if dt == torch.int32 else torch.float64
        energies = torch.empty(B, S, dtype=edt, device=J_packed.device)
        states = torch.empty(B, S, dtype=torch.int64, device=J_packed.device)
    sh = _stream_handle(stream)
    st = lib.bf_low_spectrum_batched(B, J_packed.data_ptr(), J_offsets.data_ptr(), h_packed.data_ptr(),
                                     h_offsets.data_ptr(), n.data_ptr(), n_max, S, _DTYPES[dt],
                                     energies.data_ptr(), states.data_ptr(), workspace.data_ptr(),
                                     workspace.numel(), ctypes.byref(o), sh)
    _lib.check(st, lib)
    if check:
        _lib.check(lib.bf_workspace_status(workspace.data_ptr(), sh), lib)
    return energies, states


def low_spectrum_backward(states, grad_E, n, J_offsets, h_offsets, dJ_numel: int, dh_numel: int,
                          dtype: torch.dtype = torch.float64, stream=None):
    """dL/dJ (strict upper triangles, packed like J) and dL/dh for L = sum g[b,k] E_b(states[b,k]).

    states (B, S) int64 holding uint64 configurations, grad_E (B, S) float64, n (B,) int32,
    offsets int64; returns (dJ, dh) flat tensors of the given dtype.
    """
    lib = _lib.load()
    B, S = states.shape
    dev = states.device
    dJ = torch.empty(dJ_numel, dtype=dtype, device=dev)
    dh = torch.empty(dh_numel, dtype=dtype, device=dev)
    g = grad_E.to(torch.float64).contiguous()
    st = lib.bf_low_spectrum_backward(states.contiguous().data_ptr(), g.data_ptr(), n.data_ptr(), B, S,
                                      J_offsets.data_ptr(), h_offsets.data_ptr(), dJ.data_ptr(), dh.data_ptr(),
                                      _lib.BF_F64 if dtype == torch.float64 else _lib.BF_F32,
                                      _stream_handle(stream))
    _lib.check(st, lib)
    return dJ, dh


class LowSpectrumFn(torch.autograd.Function):
    """energies, states = LowSpectrumFn.apply(J, h, S).

    Forward: the S lowest energies (float64) and configurations of one float instance.
    Backward: dL/dJ (strict upper triangle; the diagonal and lower triangle get 0, as
    they do not enter the energy) and dL/dh, computed by the backward kernel from the
    saved states.
    """

    @staticmethod
    def forward(ctx, J, h, S):
        en, st = low_spectrum(J, h, S)
        ctx.save_for_backward(st)
        ctx.n = J.shape[0]
        ctx.jdtype, ctx.hdtype = J.dtype, h.dtype
        ctx.mark_non_differentiable(st)
        return en, st

    @staticmethod
    def backward(ctx, g_en, g_st):
        (st,) = ctx.saved_tensors
        n = ctx.n
        dev = st.device
        if g_en is None:
            g_en = torch.zeros(st.shape[0], dtype=torch.float64, device=dev)
        nt = torch.tensor([n], dtype=torch.int32, device=dev)
        zero = torch.zeros(1, dtype=torch.int64, device=dev)
        dJ, dh = low_spectrum_backward(st.view(1, -1), g_en.view(1, -1), nt, zero, zero, n * n, n)
        return dJ.view(n, n).to(ctx.jdtype), dh.to(ctx.hdtype), None


class LowSpectrumBatchedFn(torch.autograd.Function):
    """energies (B, S), states = LowSpectrumBatchedFn.apply(J_packed, h_packed, J_offsets, h_offsets, n, S, n_max).

    Batched forward (bf_low_spectrum_batched) and the hand-written backward kernel;
    gradients are returned packed like J_packed and h_packed.
    """

    @staticmethod
    def forward(ctx, J_packed, h_packed, J_offsets, h_offsets, n, S, n_max):
        en, st = low_spectrum_batched(J_packed, J_offsets, h_packed, h_offsets, n, S, n_max=n_max)
        ctx.save_for_backward(st, n, J_offsets, h_offsets)
        ctx.sizes = (J_packed.numel(), h_packed.numel(), J_packed.dtype, h_packed.dtype)
        ctx.mark_non_differentiable(st)
        return en.to(torch.float64), st

    @staticmethod
    def backward(ctx, g_en, g_st):
        st, n, J_offsets, h_offsets = ctx.saved_tensors
        nj, nh, jdt, hdt = ctx.sizes
        if g_en is None:
            g_en = torch.zeros(st.shape, dtype=torch.float64, device=st.device)
        dJ, dh = low_spectrum_backward(st, g_en, n, J_offsets, h_offsets, nj, nh)
        return dJ.to(jdt), dh.to(hdt), None, None, None, None, None


def autotune_batched(J_packed, J_offsets, h_packed, h_offsets, n, S: int, *, n_max: int, stream=None):
    """Time the batched search over candidate unit sizes and grids (bf_autotune_batched).

    Returns {"task_log2", "grid_blocks", "ms"}; the choice is cached in the library for
    this device and batch shape, so later calls with default options use it.
    """
    lib = _lib.load()
    dt = J_packed.dtype
    B = n.shape[0]
    nbytes = batched_workspace_size(B, n_max, S, dt, task_log2=21)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=J_packed.device)
    edt = torch.int64 if dt == torch.int32 else torch.float64
    en = torch.empty(B, S, dtype=edt, device=J_packed.device)
    st = torch.empty(B, S, dtype=torch.int64, device=J_packed.device)
    best = _lib.Options()
    ms = ctypes.c_float(0.0)
    status = lib.bf_autotune_batched(B, J_packed.data_ptr(), J_offsets.data_ptr(), h_packed.data_ptr(),
                                     h_offsets.data_ptr(), n.data_ptr(), n_max, S, _DTYPES[dt], en.data_ptr(),
                                     st.data_ptr(), ws.data_ptr(), nbytes, _stream_handle(stream),
                                     ctypes.byref(best), ctypes.byref(ms))
    _lib.check(status, lib)
    return {"task_log2": best.task_log2, "grid_blocks": best.grid_blocks, "ms": float(ms.value)}
