"""QAOA Max-Cut energies and adjoint gradients (C ABI ``iqs_qaoa_*``).

``QAOA`` wraps one workspace (graph, qubit count, dtype, maximum batch).
``QAOAEnergy`` is a ``torch.autograd.Function`` whose forward evaluates the
energies of a batch of parameter sets and whose backward returns the adjoint
gradient computed by the CUDA engine (uncompute, no stored states).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import call, lib
from .register import _dtype_code, _stream_handle

_dp = C.POINTER(C.c_double)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


class QAOA:
    """Workspace for QAOA Max-Cut on one unweighted graph.

    ``run(gammas, betas, grad=True)`` evaluates all rows of the (batch, p)
    parameter arrays in one engine call and returns numpy arrays
    (energies[batch], d/dgamma[batch, p], d/dbeta[batch, p]).
    """

    def __init__(self, n: int, edges, dtype="complex64", batch_max: int = 1, stream=None,
                 renorm_every: int = 0, use_graphs: bool = True, *, graphs=None, per_graph: int = 0):
        """One graph (``edges``), or with ``graphs`` (a list of edge lists of
        equal length) one workspace of len(graphs) x ``per_graph`` states in
        which parameter set b is scored on graph b // per_graph."""
        self.n = int(n)
        self.dtype_code = _dtype_code(dtype)
        h = C.c_void_p()
        if graphs is None:
            e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
            self.n_edges, self.batch_max, self.n_graphs = e.shape[0], int(batch_max), 1
            call("iqs_qaoa_create", self.n, self.dtype_code, self.batch_max, self.n_edges,
                 e.ctypes.data_as(C.POINTER(C.c_int32)), _stream_handle(stream), C.byref(h))
        else:
            es = [np.asarray(g, dtype=np.int32).reshape(-1, 2) for g in graphs]
            if len({x.shape[0] for x in es}) != 1:
                raise ValueError("every graph needs the same number of edges")
            e = np.ascontiguousarray(np.concatenate(es))
            self.n_graphs, self.n_edges = len(es), es[0].shape[0]
            self.batch_max = self.n_graphs * int(per_graph)
            call("iqs_qaoa_create_multi", self.n, self.dtype_code, self.n_graphs, int(per_graph), self.n_edges,
                 e.ctypes.data_as(C.POINTER(C.c_int32)), _stream_handle(stream), C.byref(h))
        self.per_graph = self.batch_max if graphs is None else int(per_graph)
        self._h = h
        self.set_options(renorm_every, use_graphs)

    def set_engine(self, engine: str = "auto") -> None:
        """Energy-only runs: "auto", "tiled" or "cluster" (complex64 states resident on chip)."""
        call("iqs_qaoa_set_engine", self._h, {"auto": 0, "tiled": 1, "cluster": 2}[engine])

    def max_cut(self) -> np.ndarray:
        """Exact Max-Cut value of each graph (largest cut count over all bipartitions)."""
        out = np.empty(self.n_graphs)
        call("iqs_qaoa_max_cut", self._h, _ptr(out))
        return out

    def pso(self, pos0, vel0, rp, rg, omega=0.66, phi_p=1.6, phi_g=0.62):
        """Particle swarm over (gamma_1..p, beta_1..p), one swarm of per_graph
        particles per graph.  pos0, vel0: (G, R, 2p); rp, rg: (steps, G, R).
        Returns (trace (G, (steps+1) R) of best-so-far scores, best_pos (G, 2p),
        best_val (G,))."""
        x = np.ascontiguousarray(np.asarray(pos0, dtype=np.float64))
        v = np.ascontiguousarray(np.asarray(vel0, dtype=np.float64))
        a = np.ascontiguousarray(np.asarray(rp, dtype=np.float64))
        b = np.ascontiguousarray(np.asarray(rg, dtype=np.float64))
        G, R, D = x.shape
        if (G, R) != (self.n_graphs, self.per_graph) or v.shape != x.shape or D % 2:
            raise ValueError("positions must be (n_graphs, per_graph, 2p)")
        steps = a.shape[0]
        if a.shape != (steps, G, R) or b.shape != a.shape:
            raise ValueError("rp and rg must be (steps, n_graphs, per_graph)")
        trace = np.empty((G, (steps + 1) * R))
        best_pos, best_val = np.empty((G, D)), np.empty(G)
        call("iqs_qaoa_pso", self._h, D // 2, steps, _ptr(x), _ptr(v), _ptr(a), _ptr(b), C.c_double(omega),
             C.c_double(phi_p), C.c_double(phi_g), _ptr(trace), _ptr(best_pos), _ptr(best_val))
        return trace, best_pos, best_val

    def set_options(self, renorm_every: int = 0, use_graphs: bool = True) -> None:
        call("iqs_qaoa_set_options", self._h, int(renorm_every), int(bool(use_graphs)))

    def run(self, gammas, betas, grad: bool = True):
        g = np.ascontiguousarray(np.atleast_2d(np.asarray(gammas, dtype=np.float64)))
        b = np.ascontiguousarray(np.atleast_2d(np.asarray(betas, dtype=np.float64)))
        if g.shape != b.shape:
            raise ValueError("gammas and betas must have the same (batch, p) shape")
        batch, p = g.shape
        E = np.empty(batch)
        if grad:
            dg, db = np.empty((batch, p)), np.empty((batch, p))
            call("iqs_qaoa_run", self._h, batch, p, _ptr(g), _ptr(b), _ptr(E), _ptr(dg), _ptr(db))
            return E, dg, db
        call("iqs_qaoa_run", self._h, batch, p, _ptr(g), _ptr(b), _ptr(E), None, None)
        return E

    def run_async(self, gammas, betas, energies, grad_gammas=None, grad_betas=None) -> None:
        """Stream-ordered evaluation on device arrays (iqs_qaoa_run_async): ``gammas`` and ``betas``
        are contiguous float64 CUDA tensors [batch][p]; ``energies`` [batch] and, optionally,
        ``grad_gammas``/``grad_betas`` [batch][p] are float64 CUDA tensors written on the workspace's
        stream.  Returns at once; call synchronize() (or order on the stream) before reading."""
        batch, p = int(gammas.shape[0]), int(gammas.shape[1])
        dp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        call("iqs_qaoa_run_async", self._h, batch, p, dp(gammas), dp(betas), dp(energies), dp(grad_gammas),
             dp(grad_betas))

    def synchronize(self) -> None:
        """Wait for the workspace's stream; raises on a range error or a TMA wait that gave up."""
        call("iqs_qaoa_synchronize", self._h)

    def autotune(self, batch: int | None = None, p: int = 4) -> dict:
        """Pick the fastest mixer tile shape and grid size for (batch, p); returns the choice."""
        ms = C.c_double()
        call("iqs_qaoa_autotune", self._h, int(batch or self.batch_max), int(p), C.byref(ms))
        return dict(self.tuning(), best_ms=ms.value)

    def tuning(self) -> dict:
        rows, mult, tma, avail = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        call("iqs_qaoa_tuning", self._h, C.byref(rows), C.byref(mult))
        call("iqs_qaoa_get_tma", self._h, C.byref(tma), C.byref(avail))
        return {"row_bits": rows.value, "grid_mult": mult.value, "tma_mode": tma.value, "tma_available": bool(avail.value),
                **self.schedule()}

    def set_schedule(self, schedule: str = "chained") -> None:
        """Pass schedule: "chained" (segments that merge the passes at layer boundaries, the default) or
        "per_layer" (one pass sequence per layer; the only one with TMA staging)."""
        call("iqs_qaoa_set_schedule", self._h, {"chained": 0, "per_layer": 1}[schedule])

    def schedule(self) -> dict:
        sch, avail = C.c_int(), C.c_int()
        call("iqs_qaoa_get_schedule", self._h, C.byref(sch), C.byref(avail))
        return {"schedule": ("chained", "per_layer")[sch.value], "chained_available": bool(avail.value)}

    def set_tma(self, mode: int) -> None:
        """Stage mixer tiles with TMA: 0 off, 1 forward passes (the default), 2 forward and adjoint passes."""
        call("iqs_qaoa_set_tma", self._h, int(mode))

    def state(self, index: int = 0) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=np.complex128 if self.dtype_code == _lib.IQS_C128 else np.complex64)
        call("iqs_qaoa_download_state", self._h, int(index), C.c_void_p(out.ctypes.data), C.c_size_t(out.nbytes))
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.iqs_qaoa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class QAOAEnergy(torch.autograd.Function):
        """energies = QAOAEnergy.apply(gammas, betas, engine) for (batch, p) tensors.

        Forward runs the engine once; when gradients are needed it returns the
        adjoint gradient in the same call and backward scales it by the
        incoming gradient.
        """

        @staticmethod
        def forward(ctx, gammas, betas, engine: QAOA):
            need = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
            g = gammas.detach().to("cpu", torch.float64).numpy()
            b = betas.detach().to("cpu", torch.float64).numpy()
            squeeze = g.ndim == 1
            if need:
                E, dg, db = engine.run(g, b, grad=True)
                ctx.save_for_backward(torch.from_numpy(dg).to(gammas), torch.from_numpy(db).to(betas))
            else:
                E = engine.run(g, b, grad=False)
            ctx.squeeze = squeeze
            out = torch.from_numpy(E).to(device=gammas.device, dtype=torch.float64)
            return out[0] if squeeze else out

        @staticmethod
        def backward(ctx, grad_out):
            dg, db = ctx.saved_tensors
            go = grad_out.reshape(-1, 1).to(dg)
            gg, gb = go * dg, go * db
            if ctx.squeeze:
                gg, gb = gg[0], gb[0]
            return gg, gb, None

    return QAOAEnergy


def __getattr__(name):
    if name == "QAOAEnergy":
        return _autograd_function()
    raise AttributeError(name)
