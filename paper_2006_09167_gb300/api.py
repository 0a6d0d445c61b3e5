"""Python binding of the C ABI (include/nb.h): argument marshalling only.

Every compute step runs in libnb's CUDA kernels.  PyTorch supplies device
memory (tensors) and the current CUDA stream; the functions below pass raw
device pointers and the stream handle through to the library and raise
NbError for any non-OK status.  Names follow the C entry points.
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional

import numpy as np
import torch

from . import _abi
from ._abi import (NB_COULOMB_EWALD, NB_COULOMB_NONE, NB_COULOMB_RF, NB_ENERGY, NB_LIST_INNER, NB_LIST_OUTER,  # noqa: F401
                   NB_TRACE_FORCES, NB_TRACE_GATHER, NB_TRACE_KINDS, NB_TRACE_PRUNE, NB_TRACE_VJP, NB_VIRIAL, NbError,
                   check)


def _stream(stream: Optional[torch.cuda.Stream] = None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, dtype, numel: int, name: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be contiguous {dtype} with {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


class NbContext:
    """One system: wraps an nb_ctx handle (see nb_create in include/nb.h)."""

    def __init__(self, n_atoms: int, q, types, c6, c12, excl_off, excl_idx, *, coulomb: int, rc: float,
                 rlist: float, r_in: Optional[float] = None, eps_r: float = 1.0, eps_rf: float = math.inf,
                 beta: float = 0.0):
        lib = _abi.load()
        self.n = int(n_atoms)
        self.c6 = np.ascontiguousarray(c6, dtype=np.float32)
        self.c12 = np.ascontiguousarray(c12, dtype=np.float32)
        self.T = int(self.c6.shape[0])
        self.coulomb = int(coulomb)
        self.rc = float(rc)
        self.rlist = float(rlist)
        self.r_in = float(rc if r_in is None else r_in)
        p = _abi.NbParams()
        p.n_atoms = self.n
        p.n_types = self.T
        p.coulomb = self.coulomb
        p.reserved = 0
        p.eps_r = float(eps_r)
        p.eps_rf = float(eps_rf)
        p.beta = float(beta)
        p.rc = self.rc
        p.rlist = self.rlist
        p.r_in = self.r_in
        f32p = ctypes.POINTER(ctypes.c_float)
        i32p = ctypes.POINTER(ctypes.c_int32)
        p.c6_host = self.c6.ctypes.data_as(f32p)
        p.c12_host = self.c12.ctypes.data_as(f32p)
        qh = np.ascontiguousarray(q, dtype=np.float32)
        th = np.ascontiguousarray(types, dtype=np.int32)
        eo = np.ascontiguousarray(excl_off, dtype=np.int32)
        ei = np.ascontiguousarray(excl_idx, dtype=np.int32)
        if ei.size == 0:
            ei = np.zeros(1, dtype=np.int32)
        h = ctypes.c_void_p()
        check(lib.nb_create(ctypes.byref(p), qh.ctypes.data_as(f32p), th.ctypes.data_as(i32p),
                            eo.ctypes.data_as(i32p), ei.ctypes.data_as(i32p), ctypes.byref(h)),
              "nb_create")
        self.handle = h
        self.box = None
        self._lib = lib

    @classmethod
    def from_system(cls, s, r_in: Optional[float] = None) -> "NbContext":
        """Context for a synth.System (any object with the same fields)."""
        return cls(s.n, s.q, s.types, s.c6, s.c12, s.excl_off, s.excl_idx, coulomb=s.coulomb, rc=s.rc,
                   rlist=s.rlist, r_in=s.r_in if r_in is None else r_in, eps_r=s.eps_r, eps_rf=s.eps_rf,
                   beta=s.beta)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.nb_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- C entry points -------------------------------------------------
    def nb_set_charges(self, q: torch.Tensor, stream=None):
        check(self._lib.nb_set_charges(self.handle, _dev(q, torch.float32, self.n, "q"), _stream(stream)),
              "nb_set_charges")

    def nb_set_lj(self, c6: torch.Tensor, c12: torch.Tensor, stream=None):
        tt = self.T * self.T
        check(self._lib.nb_set_lj(self.handle, _dev(c6, torch.float32, tt, "c6"),
                                  _dev(c12, torch.float32, tt, "c12"), _stream(stream)), "nb_set_lj")

    def nb_grid_sort(self, x: torch.Tensor, box, stream=None):
        b = (ctypes.c_double * 3)(*[float(v) for v in box])
        check(self._lib.nb_grid_sort(self.handle, _dev(x, torch.float32, 3 * self.n, "x"), b, _stream(stream)),
              "nb_grid_sort")
        self.box = np.array([float(v) for v in box])

    def nb_pairlist_build(self, rlist: Optional[float] = None, stream=None):
        r = self.rlist if rlist is None else float(rlist)
        check(self._lib.nb_pairlist_build(self.handle, ctypes.c_float(r), _stream(stream)), "nb_pairlist_build")

    def nb_prune_rolling(self, part: int, n_parts: int, r_in: Optional[float] = None, stream=None):
        r = self.r_in if r_in is None else float(r_in)
        check(self._lib.nb_prune_rolling(self.handle, ctypes.c_float(r), int(part), int(n_parts),
                                         _stream(stream)), "nb_prune_rolling")

    def nb_forces(self, flags: int, x: torch.Tensor, f: torch.Tensor, e: Optional[torch.Tensor] = None,
                  vir: Optional[torch.Tensor] = None, stream=None):
        ep = _dev(e, torch.float64, 2, "e") if (flags & NB_ENERGY) else None
        vp = _dev(vir, torch.float64, 9, "vir") if (flags & NB_VIRIAL) else None
        check(self._lib.nb_forces(self.handle, ctypes.c_uint(flags), _dev(x, torch.float32, 3 * self.n, "x"),
                                  _dev(f, torch.float32, 3 * self.n, "f"), ep, vp, _stream(stream)), "nb_forces")

    def nb_forces_vjp_dev(self, x, gF, gE: torch.Tensor, gx, gq, gc6, gc12, stream=None):
        """nb_forces_vjp with gE a one-element float64 CUDA tensor (no host synchronisation)."""
        tt = self.T * self.T
        check(self._lib.nb_forces_vjp_dev(self.handle, _dev(x, torch.float32, 3 * self.n, "x"),
                                          _dev(gF, torch.float32, 3 * self.n, "gF"), _dev(gE, torch.float64, 1, "gE"),
                                          _dev(gx, torch.float32, 3 * self.n, "gx"),
                                          _dev(gq, torch.float32, self.n, "gq"), _dev(gc6, torch.float64, tt, "gc6"),
                                          _dev(gc12, torch.float64, tt, "gc12"), _stream(stream)), "nb_forces_vjp_dev")

    def n_slots(self) -> int:
        """Slots of the sorted layout (64 per super-cluster, padding included)."""
        return int(self.nb_get_stats()["n_slots"])

    def nb_sorted_export(self, xq: Optional[torch.Tensor] = None, perm: Optional[torch.Tensor] = None, stream=None):
        """Sorted positions and charges [n_slots, 4] and the slot -> atom permutation [n_slots]
        (-1 for padding) of the last grid sort, into the given tensors or new ones."""
        ns = self.n_slots()
        dev = torch.device("cuda", torch.cuda.current_device())
        if xq is None:
            xq = torch.empty((ns, 4), dtype=torch.float32, device=dev)
        if perm is None:
            perm = torch.empty(ns, dtype=torch.int32, device=dev)
        check(self._lib.nb_sorted_export(self.handle, _dev(xq, torch.float32, 4 * ns, "xq"),
                                         _dev(perm, torch.int32, ns, "perm"), _stream(stream)), "nb_sorted_export")
        return xq, perm

    def nb_forces_sorted(self, flags: int, xq: torch.Tensor, f: torch.Tensor, e: Optional[torch.Tensor] = None,
                         vir: Optional[torch.Tensor] = None, stream=None):
        """Forces [n_slots, 4] at the sorted positions xq [n_slots, 4] (see nb_forces_sorted)."""
        ns = self.n_slots()
        ep = _dev(e, torch.float64, 2, "e") if (flags & NB_ENERGY) else None
        vp = _dev(vir, torch.float64, 9, "vir") if (flags & NB_VIRIAL) else None
        check(self._lib.nb_forces_sorted(self.handle, ctypes.c_uint(flags), _dev(xq, torch.float32, 4 * ns, "xq"),
                                         _dev(f, torch.float32, 4 * ns, "f"), ep, vp, _stream(stream)),
              "nb_forces_sorted")

    def nb_forces_vjp(self, x, gF, gE: float, gx, gq, gc6, gc12, stream=None):
        tt = self.T * self.T
        check(self._lib.nb_forces_vjp(self.handle, _dev(x, torch.float32, 3 * self.n, "x"),
                                      _dev(gF, torch.float32, 3 * self.n, "gF"), ctypes.c_double(float(gE)),
                                      _dev(gx, torch.float32, 3 * self.n, "gx"),
                                      _dev(gq, torch.float32, self.n, "gq"), _dev(gc6, torch.float64, tt, "gc6"),
                                      _dev(gc12, torch.float64, tt, "gc12"), _stream(stream)), "nb_forces_vjp")

    def nb_count_pairs(self, which: int = NB_LIST_INNER, stream=None):
        """(pairs inside rc, atom pairs evaluated) from the inner or outer list."""
        a = ctypes.c_int64()
        b = ctypes.c_int64()
        check(self._lib.nb_count_pairs(self.handle, int(which), ctypes.byref(a), ctypes.byref(b),
                                       _stream(stream)), "nb_count_pairs")
        return a.value, b.value

    def nb_debug_export_pairs(self, which: int = NB_LIST_INNER, stream=None) -> np.ndarray:
        n = ctypes.c_size_t()
        check(self._lib.nb_debug_export_pairs(self.handle, int(which), None, 0, ctypes.byref(n), _stream(stream)),
              "nb_debug_export_pairs")
        buf = np.zeros((max(int(n.value), 1), 5), dtype=np.int64)
        check(self._lib.nb_debug_export_pairs(self.handle, int(which),
                                              buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                              buf.shape[0], ctypes.byref(n), _stream(stream)),
              "nb_debug_export_pairs")
        return buf[:n.value]

    def nb_debug_layout(self, stream=None):
        st = self.nb_get_stats()
        ns = st["n_slots"]
        perm = np.zeros(ns, dtype=np.int32)
        xq = np.zeros((ns, 4), dtype=np.float32)
        bb = np.zeros((st["n_clusters"], 8), dtype=np.float32)
        check(self._lib.nb_debug_layout(self.handle, perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                        xq.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        bb.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream(stream)),
              "nb_debug_layout")
        return perm, xq, bb

    def nb_get_stats(self) -> dict:
        s = _abi.NbStats()
        check(self._lib.nb_get_stats(self.handle, ctypes.byref(s)), "nb_get_stats")
        return {k: int(getattr(s, k)) for k, _ in _abi.NbStats._fields_}

    def nb_set_fused_prune(self, on: bool = True):
        """First prune after each list build inside the next force call (nb_set_fused_prune)."""
        check(self._lib.nb_set_fused_prune(self.handle, int(bool(on))), "nb_set_fused_prune")

    def nb_set_split(self, split: int):
        check(self._lib.nb_set_split(self.handle, int(split)), "nb_set_split")

    def nb_set_search_segments(self, segments: int):
        """Column segments of the pair search, 1..8, or 0 for the library's choice (nb_set_search_segments)."""
        check(self._lib.nb_set_search_segments(self.handle, int(segments)), "nb_set_search_segments")

    def nb_trace_enable(self, enable: bool = True, kinds=None):
        """Time launches with CUDA events: every kind (kinds=None) or the listed
        NB_TRACE_* kinds; enable=False turns tracing off."""
        mask = 0
        if enable:
            mask = (1 << NB_TRACE_KINDS) - 1 if kinds is None else sum(1 << k for k in set(kinds))
        check(self._lib.nb_trace_enable(self.handle, mask), "nb_trace_enable")

    def nb_trace_read(self, kind: int):
        """(total device ms, launches) of traced kernels of `kind` since the last read."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        check(self._lib.nb_trace_read(self.handle, int(kind), ctypes.byref(ms), ctypes.byref(n)), "nb_trace_read")
        return ms.value, n.value

    def nb_get_error(self, stream=None) -> int:
        return int(self._lib.nb_get_error(self.handle, _stream(stream)))

    def nb_ewald_corrections(self, flags: int, x: torch.Tensor, f: torch.Tensor, e: Optional[torch.Tensor] = None,
                             vir: Optional[torch.Tensor] = None, stream=None):
        """Exclusion and self terms of the Ewald sum; forces are added to f."""
        ep = _dev(e, torch.float64, 2, "e") if (flags & NB_ENERGY) else None
        vp = _dev(vir, torch.float64, 9, "vir") if (flags & NB_VIRIAL) else None
        check(self._lib.nb_ewald_corrections(self.handle, ctypes.c_uint(flags), _dev(x, torch.float32, 3 * self.n, "x"),
                                             _dev(f, torch.float32, 3 * self.n, "f"), ep, vp, _stream(stream)),
              "nb_ewald_corrections")

    # ---- conveniences ---------------------------------------------------
    def build(self, x: torch.Tensor, box, rlist: Optional[float] = None, stream=None):
        """Grid sort plus outer-list search (with the first full prune at r_in)."""
        self.nb_grid_sort(x, box, stream)
        self.nb_pairlist_build(rlist, stream)

    def forces(self, x: torch.Tensor, energy: bool = True, virial: bool = False, stream=None):
        """Returns (F [N,3] float32, E [2] float64 or None, W [3,3] float64 or None)."""
        f = torch.empty((self.n, 3), dtype=torch.float32, device=x.device)
        e = torch.empty(2, dtype=torch.float64, device=x.device) if energy else None
        w = torch.empty(9, dtype=torch.float64, device=x.device) if virial else None
        flags = (NB_ENERGY if energy else 0) | (NB_VIRIAL if virial else 0)
        self.nb_forces(flags, x.contiguous(), f, e, w, stream)
        return f, e, (w.view(3, 3) if w is not None else None)


def pme_grid(box, spacing: float = 0.12):
    """PME grid sizes: per axis the smallest even number >= L/spacing whose prime
    factors are 2, 3, 5 and 7 (sizes the FFT library handles fastest)."""
    out = []
    for L in np.asarray(box, np.float64):
        k = max(int(math.ceil(float(L) / spacing)), 8)
        while True:
            m = k
            for p in (2, 3, 5, 7):
                while m % p == 0:
                    m //= p
            if m == 1 and k % 2 == 0:
                break
            k += 1
        out.append(k)
    return tuple(out)


class NbPme:
    """Wraps an nb_pme handle (smooth PME of the reciprocal-space Ewald term)."""

    def __init__(self, n_atoms: int, beta: float, box=None, *, grid=None, spacing: float = 0.12, order: int = 4,
                 eps_r: float = 1.0):
        lib = _abi.load()
        if grid is None:
            if box is None:
                raise ValueError("give the grid or a box to size it from")
            grid = pme_grid(box, spacing)
        p = _abi.NbPmeParams()
        p.n_atoms = int(n_atoms)
        for a in range(3):
            p.grid[a] = int(grid[a])
        p.order = int(order)
        p.reserved = 0
        p.beta = float(beta)
        p.eps_r = float(eps_r)
        h = ctypes.c_void_p()
        check(lib.nb_pme_create(ctypes.byref(p), ctypes.byref(h)), "nb_pme_create")
        self.handle = h
        self._lib = lib
        self.n = int(n_atoms)
        self.grid = tuple(int(g) for g in grid)
        self.order = int(order)

    @classmethod
    def from_system(cls, s, **kw) -> "NbPme":
        return cls(s.n, s.beta, s.box, eps_r=s.eps_r, **kw)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.nb_pme_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nb_pme_forces(self, flags: int, x: torch.Tensor, q: torch.Tensor, box, f: torch.Tensor,
                      e: Optional[torch.Tensor] = None, vir: Optional[torch.Tensor] = None, stream=None):
        """Reciprocal-space forces (added to f), energy e[0] and virial."""
        b = (ctypes.c_double * 3)(*[float(v) for v in box])
        ep = _dev(e, torch.float64, 1, "e") if (flags & NB_ENERGY) else None
        vp = _dev(vir, torch.float64, 9, "vir") if (flags & NB_VIRIAL) else None
        check(self._lib.nb_pme_forces(self.handle, ctypes.c_uint(flags), _dev(x, torch.float32, 3 * self.n, "x"),
                                      _dev(q, torch.float32, self.n, "q"), b,
                                      _dev(f, torch.float32, 3 * self.n, "f"), ep, vp, _stream(stream)),
              "nb_pme_forces")


class NbBatch:
    """Wraps an nb_batch handle over several contexts (nb_batch_create)."""

    def __init__(self, ctxs):
        lib = _abi.load()
        self.ctxs = list(ctxs)
        arr = (ctypes.c_void_p * len(self.ctxs))(*[c.handle.value for c in self.ctxs])
        h = ctypes.c_void_p()
        check(lib.nb_batch_create(arr, len(self.ctxs), ctypes.byref(h)), "nb_batch_create")
        self.handle = h
        self._lib = lib
        self.offsets = np.concatenate([[0], np.cumsum([c.n for c in self.ctxs])]).astype(np.int64)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.nb_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nb_forces_batched(self, flags: int, x, f, e=None, vir=None, stream=None):
        n = int(self.offsets[-1])
        r = len(self.ctxs)
        ep = _dev(e, torch.float64, 2 * r, "e") if (flags & NB_ENERGY) else None
        vp = _dev(vir, torch.float64, 9 * r, "vir") if (flags & NB_VIRIAL) else None
        check(self._lib.nb_forces_batched(self.handle, ctypes.c_uint(flags), _dev(x, torch.float32, 3 * n, "x"),
                                          _dev(f, torch.float32, 3 * n, "f"), ep, vp, _stream(stream)),
              "nb_forces_batched")


class _ForcesFn(torch.autograd.Function):
    """F, E = forces(x, q, c6, c12) with the adjoint of nb_forces_vjp as backward."""

    @staticmethod
    def forward(ctx, x, q, c6, c12, nbctx):
        nbctx.nb_set_charges(q.detach().contiguous())
        nbctx.nb_set_lj(c6.detach().contiguous(), c12.detach().contiguous())
        f, e, _ = nbctx.forces(x.detach().contiguous(), energy=True)
        ctx.nbctx = nbctx
        ctx.save_for_backward(x)
        etot = e.sum()
        return f, etot

    @staticmethod
    def backward(ctx, gF, gE):
        (x,) = ctx.saved_tensors
        nb = ctx.nbctx
        if gF is None:
            gF = torch.zeros((nb.n, 3), dtype=torch.float32, device=x.device)
        # the energy weight stays on the device: no host synchronisation in the backward pass
        ge = (gE.detach().reshape(1).to(torch.float64) if gE is not None
              else torch.zeros(1, dtype=torch.float64, device=x.device)).contiguous()
        gx = torch.empty((nb.n, 3), dtype=torch.float32, device=x.device)
        gq = torch.empty(nb.n, dtype=torch.float32, device=x.device)
        gc6 = torch.empty((nb.T, nb.T), dtype=torch.float64, device=x.device)
        gc12 = torch.empty((nb.T, nb.T), dtype=torch.float64, device=x.device)
        nb.nb_forces_vjp_dev(x.detach().contiguous(), gF.contiguous().to(torch.float32), ge, gx, gq, gc6, gc12)
        return gx, gq, gc6.to(torch.float32), gc12.to(torch.float32), None


def forces(nbctx: NbContext, x: torch.Tensor, q: torch.Tensor, c6: torch.Tensor, c12: torch.Tensor):
    """Differentiable forces and total energy: returns (F [N,3], E scalar).

    Gradients flow to x, q and the [T,T] tables c6, c12 through the adjoint
    kernel (nb_forces_vjp); the pair list is the context's current inner list.
    """
    return _ForcesFn.apply(x, q, c6, c12, nbctx)
