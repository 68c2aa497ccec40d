"""GB300 tree-tensor-network sweep (arXiv 1905.01331) -- Python binding.

A thin layer over the C ABI of ``libttn.so`` (include/ttn.h): it marshals
arguments, and takes the library's device workspace from PyTorch's caching
allocator.  Every step of the sweep runs in the library's CUDA kernels; there
is no CPU implementation here, and a missing library raises.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _abi

PRECISIONS = {"fp64": _abi.TTN_FP64, "tf32": _abi.TTN_TF32, "tf32x3": _abi.TTN_TF32X3,
              "bf16": _abi.TTN_BF16, "bf16x3": _abi.TTN_BF16X3}


class TTNError(RuntimeError):
    pass


def instance_cost(L, chi, K=1, d0=2):
    """Relative cost of one sweep of an instance: its O(chi^4) contractions per
    layer (Sec. V) plus the top solve, from the bond dimensions alone."""
    chis = [d0]
    while len(chis) < int(round(math.log2(L))):
        chis.append(min(chi, chis[-1] ** 2))
    c = sum(chis[t + 1] * chis[t] ** 3 * (1 + 2 * K) for t in range(len(chis) - 1))
    return c + 150.0 * chis[-1] ** 3 * (1 + 2 * K)


def shard_instances(costs, world, rank):
    """Indices of the instances rank `rank` of `world` advances: the instances
    are independent (no collective on the data path), assigned longest first
    to the least loaded rank so that the slowest rank, which sets the job's
    time, carries as little as possible.  Every rank computes the same
    assignment from the same costs."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += costs[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Sweeper:
    """One or more TTN instances advanced together on the current CUDA device.

    ``models``: objects with ``Lx, Ly, o (d0 x d0), A, B (K x d0 x d0)`` (for
    example ``ttn_inputs.Model``); ``chis``: bond-dimension caps (int or list).
    The other arguments set the fields of ``ttn_options`` (include/ttn.h);
    ``lanczos_tol=0`` selects the precision's default top-solve tolerance.
    """

    def __init__(self, models, chis, per_node=False, prec="fp64", stream=None,
                 lanczos_tol=0.0, lanczos_max=48, lanczos_restarts=3,
                 polar_damping=1e-7, use_graph=True, shift=None, top_mode=0,
                 persistent=True, streams=8, polar_blocks=0, double_float=True, wait_polls=0,
                 tc_engine=0, tiles=None, recompute_ops=False, stage_streams=0):
        import torch
        self._torch = torch
        self.lib = _abi.load()
        if not isinstance(models, (list, tuple)):
            models = [models]
        if isinstance(chis, int):
            chis = [chis] * len(models)
        self.n = len(models)
        self._keep = []
        probs = (_abi.Problem * self.n)()
        for i, (m, chi) in enumerate(zip(models, chis)):
            o = np.ascontiguousarray(m.o, dtype=np.float64)
            A = np.ascontiguousarray(m.A, dtype=np.float64)
            B = np.ascontiguousarray(m.B, dtype=np.float64)
            self._keep += [o, A, B]
            d = int(round(o.shape[0] ** (1.0 / m.Ly)))
            if d ** m.Ly != o.shape[0]:
                raise TTNError(f"one-site term of dimension {o.shape[0]} is not d^Ly for Ly={m.Ly}")
            probs[i] = _abi.Problem(m.Lx, m.Ly, d, int(chi), A.shape[0], int(bool(per_node)),
                                    _ptr(o), _ptr(A), _ptr(B))
        opt = _abi.Options()
        self.lib.ttn_default_options(ctypes.byref(opt))
        opt.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        opt.lanczos_tol = lanczos_tol
        opt.lanczos_max = lanczos_max
        opt.lanczos_restarts = lanczos_restarts
        opt.polar_damping = polar_damping
        opt.use_graph = int(bool(use_graph))
        opt.persistent = 3 if persistent is True else (0 if persistent is False else int(persistent))
        opt.streams = int(streams)
        opt.polar_blocks = int(polar_blocks)
        opt.double_float = int(bool(double_float))
        opt.top_mode = int(top_mode)
        opt.wait_polls = int(wait_polls)
        opt.tc_engine = int(tc_engine)
        opt.recompute_ops = int(bool(recompute_ops))
        opt.stage_streams = int(stage_streams)
        if tiles:
            self._tiles = ctypes.create_string_buffer(bytes(tiles), len(tiles))
            opt.tiles = ctypes.cast(self._tiles, ctypes.c_void_p)
            opt.tiles_bytes = len(tiles)
        if shift is not None:
            opt.shift = float(shift)
        self.opt = opt
        nbytes = self.lib.ttn_workspace_bytes(probs, self.n, ctypes.byref(opt))
        if nbytes == 0:
            raise TTNError("ttn_workspace_bytes rejected the problems")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        rc = self.lib.ttn_create(ctypes.byref(h), probs, self.n, ctypes.byref(opt),
                                 ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                 ctypes.c_void_p(self.stream.cuda_stream))
        self.h = h
        self._check(rc, "ttn_create")
        self.per_node = bool(per_node)
        self.models = list(models)

    # -- helpers -------------------------------------------------------------
    def _check(self, rc, what):
        if rc != 0:
            msg = self.lib.ttn_last_error(self.h).decode() if self.h else ""
            raise TTNError(f"{what}: {_abi.STATUS.get(rc, rc)} {msg}")

    def chis(self, inst=0):
        nw, nv, nl = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int()
        self._check(self.lib.ttn_sizes(self.h, inst, ctypes.byref(nw), ctypes.byref(nv), ctypes.byref(nl)), "sizes")
        out = (ctypes.c_int * (nl.value + 1))()
        self._check(self.lib.ttn_chis(self.h, inst, out), "chis")
        return list(out)

    def _shapes(self, inst):
        chis = self.chis(inst)
        L = self.models[inst].Lx
        shapes = []
        for t in range(len(chis) - 1):
            s = (chis[t + 1], chis[t], chis[t])
            shapes.append(((L >> (t + 1)),) + s if self.per_node else s)
        return shapes, (chis[-1], chis[-1])

    # -- API -----------------------------------------------------------------
    def set_isometries(self, inst, ws, V):
        flat = np.ascontiguousarray(np.concatenate([np.asarray(w, np.float64).ravel() for w in ws]))
        v = np.ascontiguousarray(np.asarray(V, np.float64))
        self._check(self.lib.ttn_set_isometries(self.h, inst, _ptr(flat), _ptr(v)), "set_isometries")

    def get_isometries(self, inst=0):
        shapes, vs = self._shapes(inst)
        n = sum(int(np.prod(s)) for s in shapes)
        flat = np.empty(n)
        V = np.empty(vs)
        self._check(self.lib.ttn_get_isometries(self.h, inst, _ptr(flat), _ptr(V)), "get_isometries")
        ws, off = [], 0
        for s in shapes:
            k = int(np.prod(s))
            ws.append(flat[off:off + k].reshape(s))
            off += k
        return ws, V

    def _sweep_status(self, rc, strict):
        # TTN_ENOCONV from ttn_sweep: the last top solve missed its tolerance;
        # the tensors are a valid updated state (usual in the first sweeps)
        self.top_converged = rc != _abi.TTN_ENOCONV_CODE
        if rc == _abi.TTN_ENOCONV_CODE and not strict:
            return
        self._check(rc, "sweep")

    def sweep(self, n_sweeps=1, strict=False):
        """Run sweeps; returns energies of shape (n_sweeps, n_instances).
        ``self.top_converged`` tells whether the last top solves met their
        tolerance (with ``strict`` a miss raises)."""
        E = np.empty((n_sweeps, self.n))
        self._sweep_status(self.lib.ttn_sweep(self.h, n_sweeps, _ptr(E)), strict)
        return E

    def sweep_async(self, n_sweeps=1, strict=False):
        """Run sweeps without reading the energies back."""
        self._sweep_status(self.lib.ttn_sweep(self.h, n_sweeps, None), strict)

    def sweep_until(self, tol=1e-10, max_sweeps=1000):
        """Sweep until the energy per spin of every instance changes by less
        than ``tol`` between sweeps (Sec. IV), at most ``max_sweeps``.
        Returns (converged, energies of shape (sweeps run, n_instances))."""
        E = np.empty((max_sweeps, self.n))
        done = ctypes.c_int()
        rc = self.lib.ttn_sweep_until(self.h, float(tol), int(max_sweeps), ctypes.byref(done), _ptr(E))
        if rc not in (0, _abi.TTN_ENOCONV_CODE):
            self._check(rc, "sweep_until")
        return rc == 0, E[:done.value].copy()

    def autotune(self, reps=3):
        """Time the candidate tile widths, engines and split counts of every
        product shape during one sweep and keep the fastest; returns the
        table as bytes (for ``tiles=`` of another Sweeper)."""
        n = ctypes.c_size_t()
        self._check(self.lib.ttn_autotune(self.h, int(reps), None, ctypes.byref(n)), "autotune")
        buf = ctypes.create_string_buffer(n.value)
        self._check(self.lib.ttn_autotune(self.h, 0, buf, ctypes.byref(n)), "autotune export")
        return bytes(buf.raw[:n.value])

    def diagnostics(self, inst=0):
        """Isometry defect, density-matrix traces and symmetry, norm of v,
        last energy change per spin, top-solve convergence (FP64, device)."""
        out = np.zeros(10)
        self._check(self.lib.ttn_diagnostics(self.h, inst, _ptr(out), 10), "diagnostics")
        keys = ["isometry_defect", "trace_error", "asymmetry", "norm_error", "delta_e",
                "top_converged", "krylov_dim", "polar_unconverged", "polar_short_layers",
                "polar_first_try_layers"]
        return dict(zip(keys, out.tolist()))

    def energy(self, inst=0):
        E = ctypes.c_double()
        self._check(self.lib.ttn_energy(self.h, inst, ctypes.byref(E)), "energy")
        return E.value

    def ascend(self, inst, site_layer, prec=None):
        """Operators of a site layer ascended through the current isometries:
        array [site][1+2K][chi][chi] holding (o - c I, A_k, B_k) coarse-grained."""
        p = self.opt.prec if prec is None else (PRECISIONS[prec] if isinstance(prec, str) else prec)
        chis = self.chis(inst)
        K = self.models[inst].A.shape[0]
        S = (self.models[inst].Lx >> site_layer) if self.per_node else 1
        out = np.empty((S, 1 + 2 * K, chis[site_layer], chis[site_layer]))
        self._check(self.lib.ttn_ascend(self.h, inst, site_layer, p, _ptr(out)), "ascend")
        return out

    def rdm(self, inst, site_layer, which=0):
        n = self.chis(inst)[site_layer]
        out = np.empty((n, n))
        self._check(self.lib.ttn_rdm(self.h, inst, site_layer, which, _ptr(out)), "rdm")
        return out

    def env(self, inst, layer, out=None):
        """dE/dw of one isometry layer as a CUDA float64 tensor."""
        shapes, _ = self._shapes(inst)
        torch = self._torch
        if out is None:
            out = torch.empty(shapes[layer], dtype=torch.float64, device="cuda")
        self._check(self.lib.ttn_env(self.h, inst, layer, ctypes.c_void_p(out.data_ptr())), "env")
        return out

    def get_state(self):
        n = ctypes.c_size_t()
        self._check(self.lib.ttn_get_state(self.h, None, ctypes.byref(n)), "state size")
        buf = ctypes.create_string_buffer(n.value)
        self._check(self.lib.ttn_get_state(self.h, buf, ctypes.byref(n)), "get_state")
        return bytes(buf.raw)

    def set_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        self._check(self.lib.ttn_set_state(self.h, buf, len(data)), "set_state")

    def profile_sweep(self):
        """One eagerly launched sweep with every product timed by CUDA events."""
        out = np.zeros(19)
        self._check(self.lib.ttn_profile_sweep(self.h, _ptr(out), 19), "profile_sweep")
        keys = ["fp64_ms", "fp64_flops", "fp64_launches", "tc_ms", "tc_flops", "tc_launches",
                "other_ms", "other_launches", "total_ms", "df_ms", "df_flops", "df_launches",
                "dfc_ms", "dfc_flops", "dfc_launches", "fp64_bytes", "tc_bytes", "top_ms",
                "top_launches"]
        return dict(zip(keys, out.tolist()))

    @property
    def launch_count(self):
        return int(self.lib.ttn_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.ttn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
