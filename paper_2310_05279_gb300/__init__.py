"""GB300-native D3(BJ) dispersion: energy, forces and virial on the GPU.

Python binding of the C ABI in ``include/d3gb.h`` (argument marshalling only;
every step of the computation runs in the CUDA library ``libd3gb.so``).
PyTorch provides device memory and the current CUDA stream.

    from paper_2310_05279_gb300 import D3, workloads
    b = workloads.bilayer_ab_64()
    d3 = D3(b.tables, precision="mixed")
    out = d3.compute_batch(pos_cuda, types_cuda, b.offsets, b.cells, b.pbc)

Method: Ying & Fan, arXiv 2310.05279, Sec. II A (Eqs. 1-7).
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _lib
from .workloads import PBE_BJ, Tables  # noqa: F401

BOHR_A = 0.529177210903


class D3Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _params_struct(params: dict, precision: str, skin: float) -> _lib.D3Params:
    p = dict(PBE_BJ)
    p.update(params or {})
    prec = {"mixed": _lib.D3_MIXED, "fp64": _lib.D3_FP64}[precision]
    return _lib.D3Params(float(p["s6"]), float(p["s8"]), float(p["a1"]), float(p["a2"]), float(p["k1"]),
                         float(p["k2"]), float(p["k3"]), float(p["rc_disp"]), float(p["rc_cn"]), float(skin), prec)


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _host(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _dptr(t) -> int:
    return int(t.data_ptr())


class D3:
    """A library handle: tables and parameters live on the current CUDA device."""

    def __init__(self, tables: Tables, params: Optional[dict] = None, precision: str = "mixed", skin: float = 0.0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("D3 needs a CUDA device (there is no CPU fallback)")
        self.lib = _lib.load()
        self.precision = precision
        self.params = dict(PBE_BJ)
        self.params.update(params or {})
        self._p = _params_struct(self.params, precision, skin)
        self._hold = [np.ascontiguousarray(tables.nref, np.int32), np.ascontiguousarray(tables.cn_ref, np.float64),
                      np.ascontiguousarray(tables.c6_ref, np.float64), np.ascontiguousarray(tables.rcov, np.float64),
                      np.ascontiguousarray(tables.sqrtq, np.float64)]
        nref, cn, c6, rc, sq = self._hold
        self._t = _lib.D3Tables(int(nref.shape[0]), int(cn.shape[1]), nref.ctypes.data_as(_lib._ip),
                                cn.ctypes.data_as(_lib._dp), c6.ctypes.data_as(_lib._dp),
                                rc.ctypes.data_as(_lib._dp), sq.ctypes.data_as(_lib._dp))
        torch.cuda.current_device()  # initialise the primary context before the library uses it
        h = C.c_void_p()
        st = self.lib.d3_create(C.byref(self._p), C.byref(self._t), C.byref(h))
        if st != 0:
            raise D3Error(st, "d3_create failed")
        self.h = h
        if float(self.params.get("s9", 0.0)) != 0.0:  # optional three-body term
            self.set_three_body(self.params["s9"], self.params.get("alpha9", 16.0), self.params.get("rc3"))

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.d3_destroy(h)
            self.h = None

    def _check(self, st: int):
        if st != 0:
            msg = self.lib.d3_last_error(self.h)
            raise D3Error(st, msg.decode() if msg else "")

    def set_damping(self, s6: float, s8: float, a1: float, a2: float):
        self._check(self.lib.d3_set_damping(self.h, float(s6), float(s8), float(a1), float(a2)))
        self.params.update(s6=float(s6), s8=float(s8), a1=float(a1), a2=float(a2))

    @staticmethod
    def _geom(offsets, cells, pbc):
        offsets = _host(offsets, np.int64)
        B = offsets.shape[0] - 1
        cells = _host(cells, np.float64).reshape(B, 9) if B > 0 else np.zeros((0, 9))
        pbc = _host(pbc, np.int32).reshape(B, 3) if B > 0 else np.zeros((0, 3), np.int32)
        return B, offsets, cells, pbc

    def compute_batch(self, pos, types, offsets, cells, pbc, e_atom: bool = False, cn: bool = False,
                      w_atom: bool = False, out=None, stream=None) -> dict:
        """pos: cuda float64 (N,3) in A; types: cuda int32 (N,); offsets/cells/pbc: host arrays.
        Returns cuda tensors E (B,) eV, F (N,3) eV/A, W (B,3,3) eV [, e_atom (N,), cn (N,),
        w_atom (N,3,3) eV: the per-atom virial of Eq. 7]."""
        import torch
        B, offsets, cells, pbc = self._geom(offsets, cells, pbc)
        N = int(offsets[-1])
        dev = pos.device
        assert pos.is_cuda and pos.dtype == torch.float64 and pos.is_contiguous() and tuple(pos.shape) == (N, 3)
        assert types.is_cuda and types.dtype == torch.int32 and types.is_contiguous() and types.numel() == N
        if out is None:
            out = dict(E=torch.empty(B, dtype=torch.float64, device=dev),
                       F=torch.empty((N, 3), dtype=torch.float64, device=dev),
                       W=torch.empty((B, 3, 3), dtype=torch.float64, device=dev))
            if e_atom:
                out["e_atom"] = torch.empty(N, dtype=torch.float64, device=dev)
            if cn:
                out["cn"] = torch.empty(N, dtype=torch.float64, device=dev)
            if w_atom:
                out["w_atom"] = torch.empty((N, 3, 3), dtype=torch.float64, device=dev)
        ea = out.get("e_atom")
        cnv = out.get("cn")
        wa = out.get("w_atom")
        if wa is not None:
            st = self.lib.d3_compute_batch_atoms(self.h, B, offsets.ctypes.data_as(_lib._lp), _dptr(pos),
                                                 _dptr(types), cells.ctypes.data_as(_lib._dp),
                                                 pbc.ctypes.data_as(_lib._ip), _dptr(out["E"]), _dptr(out["F"]),
                                                 _dptr(out["W"]), _dptr(ea) if ea is not None else None,
                                                 _dptr(cnv) if cnv is not None else None, _dptr(wa),
                                                 _stream_ptr(stream))
            self._check(st)
            return out
        st = self.lib.d3_compute_batch_ex(self.h, B, offsets.ctypes.data_as(_lib._lp), _dptr(pos), _dptr(types),
                                          cells.ctypes.data_as(_lib._dp), pbc.ctypes.data_as(_lib._ip),
                                          _dptr(out["E"]), _dptr(out["F"]), _dptr(out["W"]),
                                          _dptr(ea) if ea is not None else None,
                                          _dptr(cnv) if cnv is not None else None, _stream_ptr(stream))
        self._check(st)
        return out

    def compute(self, pos, types, cell, pbc, stream=None) -> dict:
        """One structure (d3_compute)."""
        import torch
        n = int(pos.shape[0])
        dev = pos.device
        out = dict(E=torch.empty(1, dtype=torch.float64, device=dev),
                   F=torch.empty((n, 3), dtype=torch.float64, device=dev),
                   W=torch.empty((3, 3), dtype=torch.float64, device=dev))
        cell = _host(cell, np.float64).reshape(9)
        pbc = _host(pbc, np.int32).reshape(3)
        st = self.lib.d3_compute(self.h, _dptr(pos), _dptr(types), n, cell.ctypes.data_as(_lib._dp),
                                 pbc.ctypes.data_as(_lib._ip), _dptr(out["E"]), _dptr(out["F"]), _dptr(out["W"]),
                                 _stream_ptr(stream))
        self._check(st)
        return out

    def compute_batch_host(self, pos, types, offsets, cells, pbc, out=None, stream=None) -> dict:
        """All arrays in host memory (numpy; page-locked tensors work too); synchronises."""
        B, offsets, cells, pbc = self._geom(offsets, cells, pbc)
        N = int(offsets[-1])
        if out is None:
            out = dict(E=np.empty(B), F=np.empty((N, 3)), W=np.empty((B, 3, 3)))

        def ptr(a):
            return a.ctypes.data if isinstance(a, np.ndarray) else int(a.data_ptr())
        st = self.lib.d3_compute_batch_host(self.h, B, offsets.ctypes.data_as(_lib._lp), ptr(pos), ptr(types),
                                            cells.ctypes.data_as(_lib._dp), pbc.ctypes.data_as(_lib._ip),
                                            ptr(out["E"]), ptr(out["F"]), ptr(out["W"]), _stream_ptr(stream))
        self._check(st)
        return out

    def build_neighbors(self, pos, types, offsets, cells, pbc, stream=None):
        B, offsets, cells, pbc = self._geom(offsets, cells, pbc)
        self._check(self.lib.d3_build_neighbors(self.h, B, offsets.ctypes.data_as(_lib._lp), _dptr(pos),
                                                _dptr(types), cells.ctypes.data_as(_lib._dp),
                                                pbc.ctypes.data_as(_lib._ip), _stream_ptr(stream)))

    def backward(self, pos, types, offsets, cells, pbc, dLdE, dLdF, want_params=True, want_pos=True,
                 stream=None) -> dict:
        """dL/d(s6, s8, a1, a2[bohr]) and dL/dx for upstream dL/dE (B,) and dL/dF (N,3) (cuda float64)."""
        import torch
        B, offsets, cells, pbc = self._geom(offsets, cells, pbc)
        N = int(offsets[-1])
        dev = pos.device
        gp = torch.empty(4, dtype=torch.float64, device=dev) if want_params else None
        gx = torch.empty((N, 3), dtype=torch.float64, device=dev) if want_pos else None
        st = self.lib.d3_backward(self.h, B, offsets.ctypes.data_as(_lib._lp), _dptr(pos), _dptr(types),
                                  cells.ctypes.data_as(_lib._dp), pbc.ctypes.data_as(_lib._ip),
                                  _dptr(dLdE.contiguous()), _dptr(dLdF.contiguous()),
                                  _dptr(gp) if gp is not None else None, _dptr(gx) if gx is not None else None,
                                  _stream_ptr(stream))
        self._check(st)
        return dict(dparams=gp, dpos=gx)

    STAGES = ("build", "cn", "weights", "disp", "three_body", "chain", "finalize")

    def profile(self, on: bool = True):
        """Bracket every stage of later calls with CUDA events (see d3_profile_enable)."""
        self._check(self.lib.d3_profile_enable(self.h, 1 if on else 0))

    def profile_read(self) -> dict:
        ms = (C.c_double * len(self.STAGES))()
        calls = (C.c_int64 * len(self.STAGES))()
        launches = C.c_int64()
        self._check(self.lib.d3_profile_read(self.h, ms, calls, C.byref(launches)))
        return dict(ms={k: ms[i] for i, k in enumerate(self.STAGES)},
                    calls={k: calls[i] for i, k in enumerate(self.STAGES)}, launches=launches.value)

    def profile_reset(self):
        self._check(self.lib.d3_profile_reset(self.h))

    def sync_status(self):
        self._check(self.lib.d3_sync_status(self.h))

    def set_graphs(self, on: bool = True):
        """Replay repeated compute calls as one CUDA graph (default on)."""
        self._check(self.lib.d3_set_graphs(self.h, 1 if on else 0))

    SHAPE_KEYS = ("cn_block", "disp_block", "chain_block", "build_blocks_per_sm")

    def set_autotune(self, on: bool = True):
        """Measure the launch shapes once per size class when a new geometry is sized (default on)."""
        self._check(self.lib.d3_set_autotune(self.h, 1 if on else 0))

    def launch_shapes(self) -> dict:
        """Launch shapes used for the next call, and the number of autotuner measurements so far."""
        sh = (C.c_int32 * 4)()
        n = C.c_int64()
        self._check(self.lib.d3_launch_shapes(self.h, sh, C.byref(n)))
        return dict(zip(self.SHAPE_KEYS, list(sh)), tunings=n.value)

    def set_launch_shapes(self, cn_block: int, disp_block: int, chain_block: int, build_blocks_per_sm: int):
        """Fix the launch shapes (64 or 128 threads per pass block, 8 or 16 builder blocks per SM);
        turns autotuning off."""
        sh = (C.c_int32 * 4)(cn_block, disp_block, chain_block, build_blocks_per_sm)
        self._check(self.lib.d3_set_launch_shapes(self.h, sh))

    def set_three_body(self, s9: float = 1.0, alpha9: float = 16.0, rc3: Optional[float] = None):
        """Optional triple-dipole term that the paper leaves out (d3_set_three_body): s9 = 0 turns it
        off; rc3 (A, default R_cn) bounds every side of a triangle and may not exceed R_cn."""
        rc3 = float(self.params["rc_cn"]) if rc3 is None else float(rc3)
        self._check(self.lib.d3_set_three_body(self.h, float(s9), float(alpha9), rc3))
        self.params.update(s9=float(s9), alpha9=float(alpha9), rc3=rc3)

    def set_accumulate(self, on: bool = True):
        """Add E, F, W into the output tensors instead of overwriting them (Eq. 9 coupling)."""
        self._check(self.lib.d3_set_accumulate(self.h, 1 if on else 0))

    def profile_stage(self, stage: int):
        """(ms, calls) of one profiled stage; stage 7 is the list-builder kernel alone."""
        ms = C.c_double()
        calls = C.c_int64()
        self._check(self.lib.d3_profile_stage(self.h, int(stage), C.byref(ms), C.byref(calls)))
        return ms.value, calls.value

    STAT_KEYS = ("real_atoms", "image_atoms", "clusters", "cluster_list_entries", "cn_list_entries",
                 "disp_list_entries", "pairs_within_rpot", "list_mode")

    def list_stats(self) -> dict:
        """Sizes of the neighbour data of the current plan (d3_list_stats; synchronises)."""
        st = (C.c_int64 * 8)()
        self._check(self.lib.d3_list_stats(self.h, st))
        return dict(zip(self.STAT_KEYS, list(st)))

    def tune_times(self) -> dict:
        """The autotuner's last measurement (ms per stage and candidate)."""
        t = (C.c_float * 8)()
        self._check(self.lib.d3_tune_times(self.h, t))
        v = list(t)
        return {"build": v[0:2], "cn": v[2:4], "disp": v[4:6], "chain": v[6:8]}

    def build_count(self) -> int:
        """Neighbour builds executed on the device so far (synchronises)."""
        n = C.c_int64()
        self._check(self.lib.d3_build_count(self.h, C.byref(n)))
        return n.value


def heat_current(w_atom, vel, stream=None):
    """Per-atom heat current of Eq. 8, J_i = W_i . v_i (cuda float64 (N,3,3) and (N,3))."""
    import torch
    lib = _lib.load()
    n = int(w_atom.shape[0])
    assert w_atom.is_cuda and w_atom.dtype == torch.float64 and w_atom.is_contiguous() and w_atom.numel() == 9 * n
    assert vel.is_cuda and vel.dtype == torch.float64 and vel.is_contiguous() and vel.numel() == 3 * n
    J = torch.empty((n, 3), dtype=torch.float64, device=w_atom.device)
    st = lib.d3_heat_current(n, _dptr(w_atom), _dptr(vel), _dptr(J), _stream_ptr(stream))
    if st != _lib.D3_OK:
        raise D3Error(st, "d3_heat_current failed")
    return J


def peak_rates(stream=None) -> dict:
    """Measured FP32 FMA, FP64 FMA and MUFU reciprocal rates of the current device (d3_peak_rates)."""
    lib = _lib.load()
    r = (C.c_double * 3)()
    st = lib.d3_peak_rates(r, _stream_ptr(stream))
    if st != _lib.D3_OK:
        raise D3Error(st, "d3_peak_rates failed")
    return {"fp32_lane_ops_per_s": r[0], "fp64_lane_ops_per_s": r[1], "mufu_ops_per_s": r[2]}


def version() -> str:
    return _lib.load().d3_version().decode()


def _autograd_function():
    import torch

    class D3Function(torch.autograd.Function):
        """(E, F) = D3(pos; s6, s8, a1, a2) with the hand-written backward of d3_backward.

        apply(pos, theta, d3, types, offsets, cells, pbc): pos cuda float64 (N,3) [A],
        theta cuda float64 (4,) = (s6, s8, a1, a2[bohr]).  Returns E (B,) [eV] and F (N,3)
        [eV/A].  Gradients flow to pos and theta; the backward runs in the handle's
        precision (FP64 duals for an FP64 handle; for a mixed handle the forward's mixed
        arithmetic with FP32 tangents)."""

        @staticmethod
        def forward(ctx, pos, theta, d3, types, offsets, cells, pbc):
            th = [float(x) for x in theta.detach().cpu().tolist()]
            d3.set_damping(*th)
            out = d3.compute_batch(pos.detach().contiguous(), types, offsets, cells, pbc)
            ctx.d3, ctx.types, ctx.geom, ctx.theta = d3, types, (offsets, cells, pbc), th
            ctx.save_for_backward(pos)
            return out["E"], out["F"]

        @staticmethod
        def backward(ctx, gE, gF):
            (pos,) = ctx.saved_tensors
            d3 = ctx.d3
            offsets, cells, pbc = ctx.geom
            d3.set_damping(*ctx.theta)
            B = len(offsets) - 1
            if gE is None:
                gE = torch.zeros(B, dtype=torch.float64, device=pos.device)
            if gF is None:
                gF = torch.zeros_like(pos)
            g = d3.backward(pos.detach().contiguous(), ctx.types, offsets, cells, pbc, gE.contiguous(),
                            gF.contiguous())
            return g["dpos"], g["dparams"], None, None, None, None, None

    return D3Function


def __getattr__(name):
    if name == "D3Function":
        fn = _autograd_function()
        globals()["D3Function"] = fn
        return fn
    raise AttributeError(name)
