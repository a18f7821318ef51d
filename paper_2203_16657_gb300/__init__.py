"""GB300-native community integration algorithm (CIA) for network ODEs.

Python binding of libcia (include/cia.h): argument marshalling only.  Every
step of the hot path runs in the library's CUDA kernels; there is no CPU or
PyTorch fallback, and importing this package fails if libcia.so is missing.
PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import CiaError, load

__all__ = ["Plan", "Basis", "CiaError", "load", "status_string", "detect_communities"]


def status_string(status: int) -> str:
    return load().cia_status_string(int(status)).decode()


def _stream_handle(stream=None) -> ctypes.c_void_p:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype_name: str, n: int) -> ctypes.c_void_p:
    import torch
    want = getattr(torch, dtype_name)
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != want or not t.is_contiguous() or t.numel() != n:
        raise ValueError("expected a contiguous %s tensor of %d elements" % (dtype_name, n))
    return ctypes.c_void_p(t.data_ptr())


def detect_communities(rowptr, col, *, gamma=1.0, community_cost=0.0, min_size=2, max_levels=8, seed=0):
    """Community labels for step P1 that make S sparse (include/cia.h,
    cia_detect_communities): the Potts Hamiltonian with the Erdos-Renyi null
    model, optimised by local moving and aggregation on the host.  Returns
    (labels int32 with -1 for communities below min_size, report dict)."""
    lib = load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = len(rowptr) - 1
    g = _abi.Graph(n, rowptr.ctypes.data, col.ctypes.data)
    opt = _abi.DetectOptions(float(gamma), float(community_cost), int(min_size), int(max_levels), int(seed))
    labels = np.empty(n, dtype=np.int32)
    rep = _abi.DetectReport()
    _abi.check(lib.cia_detect_communities(ctypes.byref(g), ctypes.byref(opt), labels.ctypes.data,
                                          ctypes.byref(rep)))
    return labels, {name: getattr(rep, name) for name, _ in _abi.DetectReport._fields_}


def choose_partition(rowptr, col, omega, x, dt, steps=10, *, K=1.0, d_sin=(1.0,), d_cos=(0.0,),
                     precision="fp32", model="kuramoto", K2=0.0):
    """Community labels chosen by timing this library's kernels on three
    detected partitions (include/cia.h, cia_choose_partition): the S-minimal
    one, a coarser probe and the minimiser of the fitted stage-time model.
    x: host float64 initial state (original order).  Returns (labels, report)."""
    lib = load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = len(rowptr) - 1
    g = _abi.Graph(n, rowptr.ctypes.data, col.ctypes.data)
    cp = Plan._coupling(model, d_sin, d_cos, K, K2, 1.0, 0.0)
    opt = _abi.Options(_abi.PRECISION[precision], 0, 0, 0, 0, 0, 0)
    om = np.ascontiguousarray(omega, dtype=np.float64) if omega is not None else None
    xh = np.ascontiguousarray(x, dtype=np.float64)
    if len(xh) != n or (om is not None and len(om) != n):
        raise ValueError("x and omega must have n entries")
    labels = np.empty(n, dtype=np.int32)
    rep = _abi.PartitionReport()
    _abi.check(lib.cia_choose_partition(ctypes.byref(g), om.ctypes.data if om is not None else None,
                                        ctypes.byref(cp), ctypes.byref(opt), xh.ctypes.data, float(dt), int(steps),
                                        labels.ctypes.data, ctypes.byref(rep)))
    out = {}
    for name, _ in _abi.PartitionReport._fields_:
        v = getattr(rep, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    return labels, out


class Plan:
    """A CIA plan: step P1 done once, then E1 + E2 on the device every call.

    rowptr/col: symmetric CSR (host int64 / int32), labels: int32 community ids
    (-1 = no community), omega: natural frequencies (host float64).
    Coupling h(x) = sum_k d_sin[k] sin((k+1)x) + d_cos[k] cos((k+1)x), scaled by K/N;
    model="kuramoto_ho" adds the triadic term on community hyperedges, scaled by K2/N^2.
    model="cucker_smale": state [n, 4] = (s_x, s_y, v_x, v_y) per node, weight
    eta(y) = K (sigma^2 + y)^-beta; the CIA needs a basis (set_basis / learn_fit).
    model="polynomial": x' = -V'(x) + (K/N) sum_l a_ml h(x_l - x_m) with
    h(x) = sum_a poly_c[a] x^a (degree <= 4) and V'(x) = sum_j dV[j] x^j, FP64,
    omega None (Desai-Zwanzig: dV = (0, -1, 0, 1), poly_c = (0, 1)).
    model="polynomial_general": the same with g(x_l, x_m) = sum_{a,b} poly_g[a][b] x_l^a x_m^b,
    poly_g a square (p+1) x (p+1) array.
    model="fourier_general": the same with the real 2-D Fourier series of eq.
    FourierRealExpansion, fourier_C = (C11, C12, C21, C22) of shape (p+1) x (p+1),
    frequencies pi a / fourier_L.
    """

    def __init__(self, rowptr, col, labels, omega=None, *, K=1.0, d_sin=(1.0,), d_cos=(0.0,),
                 precision="fp64", build_direct=False, tile_nodes=0, group_size=0,
                 tile_index_bytes=0, staging="auto", model="kuramoto", K2=0.0, sigma=1.0,
                 beta=0.0, poly_c=(0.0, 1.0), dV=(0.0,), poly_g=None, fourier_L=None, fourier_C=None,
                 use_graphs=True, _batch=None):
        lib = load()
        self._lib = lib
        self._keep = []
        cp = self._coupling(model, d_sin, d_cos, K, K2, sigma, beta, poly_c, dV, poly_g, fourier_L, fourier_C)
        opt = _abi.Options(_abi.PRECISION[precision], int(bool(build_direct)), int(tile_nodes),
                           int(group_size), int(tile_index_bytes), _abi.STAGING[staging],
                           0 if use_graphs else 1)
        handle = ctypes.c_void_p()
        if _batch is not None:
            graphs, labs, oms = _batch
            B = len(graphs)
            garr = (_abi.Graph * B)()
            larr = (ctypes.c_void_p * B)()
            oarr = (ctypes.c_void_p * B)()
            keep = []
            n = 0
            for i, ((rp, cl), lb, om) in enumerate(zip(graphs, labs, oms)):
                rp = np.ascontiguousarray(rp, dtype=np.int64)
                cl = np.ascontiguousarray(cl, dtype=np.int32)
                lb = np.ascontiguousarray(lb, dtype=np.int32)
                if len(lb) != len(rp) - 1:
                    raise ValueError("instance %d: labels must have n entries" % i)
                garr[i] = _abi.Graph(len(rp) - 1, rp.ctypes.data, cl.ctypes.data)
                larr[i] = lb.ctypes.data
                keep += [rp, cl, lb]
                if om is not None:
                    om = np.ascontiguousarray(om, dtype=np.float64)
                    if len(om) != len(rp) - 1:
                        raise ValueError("instance %d: omega must have n entries" % i)
                    oarr[i] = om.ctypes.data
                    keep.append(om)
                n += len(rp) - 1
            _abi.check(lib.cia_plan_create_batch(B, garr, larr, oarr, ctypes.byref(cp),
                                                 ctypes.byref(opt), ctypes.byref(handle)))
        else:
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            labels = np.ascontiguousarray(labels, dtype=np.int32)
            n = len(rowptr) - 1
            if len(labels) != n:
                raise ValueError("labels must have n entries")
            g = _abi.Graph(n, rowptr.ctypes.data, col.ctypes.data)
            om = None
            if omega is not None:
                om = np.ascontiguousarray(omega, dtype=np.float64)
                if len(om) != n:
                    raise ValueError("omega must have n entries")
            _abi.check(lib.cia_plan_create(ctypes.byref(g), labels.ctypes.data,
                                           om.ctypes.data if om is not None else None,
                                           ctypes.byref(cp), ctypes.byref(opt), ctypes.byref(handle)))
        self._h = handle
        self.n = n
        self.precision = precision
        self.dim = 4 if model == "cucker_smale" else 1
        self.size = n * self.dim
        self.instances = self.info()["instances"]

    @classmethod
    def batch(cls, graphs, labels, omegas=None, **kw):
        """An ensemble of independent networks: graphs = [(rowptr, col), ...],
        labels and omegas per instance; states concatenate the instances and
        order parameters come as [steps, B] (include/cia.h, cia_plan_create_batch)."""
        if omegas is None:
            omegas = [None] * len(graphs)
        return cls(None, None, None, _batch=(list(graphs), list(labels), list(omegas)), **kw)

    @classmethod
    def streamed(cls, instances, *, K=1.0, d_sin=(1.0,), d_cos=(0.0,), precision="fp32", tile_nodes=0,
                 tile_index_bytes=0, staging="auto", use_graphs=True):
        """An ensemble planned one instance at a time (include/cia.h,
        cia_plan_batch_begin/add/finish): `instances` yields (rowptr, col,
        labels, omega) per instance, omega may be None; each instance's arrays
        can be dropped once the next one is requested."""
        lib = load()
        cp = cls._coupling("kuramoto", d_sin, d_cos, K, 0.0, 1.0, 0.0)
        opt = _abi.Options(_abi.PRECISION[precision], 0, int(tile_nodes), 0, int(tile_index_bytes),
                           _abi.STAGING[staging], 0 if use_graphs else 1)
        handle = ctypes.c_void_p()
        _abi.check(lib.cia_plan_batch_begin(ctypes.byref(cp), ctypes.byref(opt), ctypes.byref(handle)))
        self = cls.__new__(cls)
        self._lib = lib
        self._keep = []
        self._h = handle
        n = 0
        for rowptr, col, labels, omega in instances:
            rp = np.ascontiguousarray(rowptr, dtype=np.int64)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            lb = np.ascontiguousarray(labels, dtype=np.int32)
            if len(lb) != len(rp) - 1:
                raise ValueError("labels must have n entries")
            om = None
            if omega is not None:
                om = np.ascontiguousarray(omega, dtype=np.float64)
                if len(om) != len(rp) - 1:
                    raise ValueError("omega must have n entries")
            g = _abi.Graph(len(rp) - 1, rp.ctypes.data, cl.ctypes.data)
            _abi.check(lib.cia_plan_batch_add(handle, ctypes.byref(g), lb.ctypes.data,
                                              om.ctypes.data if om is not None else None))
            n += len(rp) - 1
        _abi.check(lib.cia_plan_batch_finish(handle))
        self.n = n
        self.precision = precision
        self.dim = 1
        self.size = n
        self.instances = self.info()["instances"]
        return self

    @staticmethod
    def _coupling(model, d_sin, d_cos, K, K2, sigma, beta, poly_c=(0.0, 1.0), dV=(0.0,), poly_g=None,
                  fourier_L=None, fourier_C=None):
        d_sin = list(d_sin)
        d_cos = list(d_cos)
        p = len(d_sin)
        poly = model in ("polynomial", "polynomial_general", "fourier_general")
        if not poly and (len(d_cos) != p or not 1 <= p <= _abi.CIA_MAX_HARMONICS):
            raise ValueError("d_sin and d_cos must have the same length in [1, %d]"
                             % _abi.CIA_MAX_HARMONICS)
        cp = _abi.Coupling()
        cp.model = _abi.MODEL[model]
        cp.p = p
        for k in range(p):
            cp.d_sin[k] = float(d_sin[k])
            cp.d_cos[k] = float(d_cos[k])
        cp.K = float(K)
        cp.K2 = float(K2)
        cp.sigma = float(sigma)
        cp.beta = float(beta)
        if poly:
            S = _abi.CIA_MAX_POLY + 1
            dV = list(dV)
            if len(dV) > S:
                raise ValueError("dV takes at most %d coefficients" % S)
            for j, v in enumerate(dV):
                cp.dV[j] = float(v)
            if model == "fourier_general":
                if fourier_L is None or fourier_C is None or len(fourier_C) != 4:
                    raise ValueError("fourier_general needs fourier_L and fourier_C = (C11, C12, C21, C22)")
                C = [np.asarray(c, dtype=np.float64) for c in fourier_C]
                q = C[0].shape[0] - 1
                if any(c.shape != (q + 1, q + 1) for c in C) or not 1 <= q <= _abi.CIA_MAX_HARMONICS:
                    raise ValueError("fourier_C must hold four (p+1) x (p+1) arrays, 1 <= p <= %d"
                                     % _abi.CIA_MAX_HARMONICS)
                cp.p = q
                cp.fourier_L = float(fourier_L)
                SH = _abi.CIA_MAX_HARMONICS + 1
                for i, c in enumerate(C):
                    for a_ in range(q + 1):
                        for b_ in range(q + 1):
                            cp.fourier_c[i][a_ * SH + b_] = float(c[a_, b_])
            elif model == "polynomial":
                poly_c = list(poly_c)
                if not 1 <= len(poly_c) <= S:
                    raise ValueError("poly_c needs 1..%d coefficients" % S)
                cp.p = len(poly_c) - 1
                for a, v in enumerate(poly_c):
                    cp.poly_c[a] = float(v)
            else:
                G = np.asarray(poly_g, dtype=np.float64) if poly_g is not None else None
                if G is None or G.ndim != 2 or G.shape[0] != G.shape[1] or not 1 <= G.shape[0] <= S:
                    raise ValueError("poly_g must be a square (p+1) x (p+1) array, p <= %d" % (S - 1))
                cp.p = G.shape[0] - 1
                for a in range(G.shape[0]):
                    for b in range(G.shape[1]):
                        cp.poly_g[a * S + b] = float(G[a, b])
        return cp

    # ------------------------------------------------------------ bookkeeping
    def info(self) -> dict:
        inf = _abi.PlanInfo()
        _abi.check(self._lib.cia_plan_get_info(self._h, ctypes.byref(inf)))
        return {name: getattr(inf, name) for name, _ in _abi.PlanInfo._fields_}

    def permutation(self):
        inf = self.info()
        perm = np.empty(self.n, dtype=np.int32)
        off = np.empty(inf["M"] + 1, dtype=np.int64)
        _abi.check(self._lib.cia_plan_get_permutation(self._h, perm.ctypes.data, off.ctypes.data))
        return perm, off

    def split(self):
        inf = self.info()
        n = self.n
        mrp = np.empty(n + 1, dtype=np.int64)
        mcol = np.empty(max(1, inf["nnz_missing"]), dtype=np.int32)
        irp = np.empty(n + 1, dtype=np.int64)
        icol = np.empty(max(1, inf["nnz_inter"]), dtype=np.int32)
        _abi.check(self._lib.cia_plan_get_split(self._h, mrp.ctypes.data, mcol.ctypes.data,
                                                irp.ctypes.data, icol.ctypes.data))
        return mrp, mcol[:inf["nnz_missing"]], irp, icol[:inf["nnz_inter"]]

    # ------------------------------------------------------------ evaluation
    def rhs(self, x, out=None, method="cia", stream=None):
        """dx/dt for x (CUDA float64, original order); returns `out`."""
        import torch
        if out is None:
            out = torch.empty_like(x)
        fn = self._lib.cia_rhs if method == "cia" else self._lib.cia_rhs_direct
        _abi.check(fn(self._h, _dev_ptr(x, "float64", self.size), _dev_ptr(out, "float64", self.size),
                      _stream_handle(stream)))
        return out

    def integrate(self, x, dt, steps, method="cia", r_out=None, stream=None):
        """Advance x (CUDA float64, original order) in place by `steps` RK4 steps."""
        rp = _dev_ptr(r_out, "float64", int(steps) * self.instances) if r_out is not None else None
        st = self._lib.cia_integrate(self._h, _abi.METHOD[method],
                                     _dev_ptr(x, "float64", self.size), float(dt), int(steps),
                                     rp, _stream_handle(stream))
        self._status(st)
        return x

    def integrate_host(self, x: np.ndarray, dt, steps, method="cia", r_out=None, stream=None):
        """Host-buffer integration (copies inside the call); x is updated in place."""
        if x.dtype != np.float64 or not x.flags.c_contiguous or x.size != self.size:
            raise ValueError("x must be a contiguous float64 array of n x d entries")
        rp = None
        if r_out is not None:
            if r_out.dtype != np.float64 or r_out.size != steps * self.instances:
                raise ValueError("r_out must be float64 with steps x instances entries")
            rp = r_out.ctypes.data
        self._status(self._lib.cia_integrate_host(self._h, _abi.METHOD[method], x.ctypes.data,
                                                  float(dt), int(steps), rp,
                                                  _stream_handle(stream)))
        return x

    def state_load(self, x, stream=None):
        """Make x (CUDA float64, original order) the resident state."""
        _abi.check(self._lib.cia_state_load(self._h, _dev_ptr(x, "float64", self.size),
                                            _stream_handle(stream)))

    def state_store(self, x, stream=None):
        """Copy the resident state into x (CUDA float64, original order)."""
        _abi.check(self._lib.cia_state_store(self._h, _dev_ptr(x, "float64", self.size),
                                             _stream_handle(stream)))
        return x

    def advance(self, dt, steps, method="cia", r_out=None, stream=None):
        """Advance the resident state by `steps` RK4 steps."""
        rp = _dev_ptr(r_out, "float64", int(steps) * self.instances) if r_out is not None else None
        self._status(self._lib.cia_advance(self._h, _abi.METHOD[method], float(dt), int(steps), rp,
                                           _stream_handle(stream)))

    def set_weights(self, alpha=None, beta=None):
        """Rank-one link weights alpha_m beta_l for the polynomial models (host
        arrays of n entries, original order; None = ones; both None removes
        them).  Load a state again before advance."""
        arrs = []
        for v in (alpha, beta):
            if v is None:
                arrs.append(None)
                continue
            v = np.ascontiguousarray(v, dtype=np.float64)
            if v.shape != (self.n,):
                raise ValueError("weights must have n entries")
            arrs.append(v)
        ptr = [a.ctypes.data if a is not None else None for a in arrs]
        _abi.check(self._lib.cia_plan_set_weights(self._h, ptr[0], ptr[1]))

    def retile(self, tile_nodes=0, tile_index_bytes=0, staging="auto"):
        _abi.check(self._lib.cia_plan_retile(self._h, int(tile_nodes), int(tile_index_bytes),
                                             _abi.STAGING[staging]))

    def autotune(self, x, dt, steps=10, stream=None) -> dict:
        """Time the candidate tilings from state x and keep the fastest."""
        r = _abi.TuneReport()
        _abi.check(self._lib.cia_plan_autotune(self._h, _dev_ptr(x, "float64", self.size), float(dt),
                                               int(steps), ctypes.byref(r), _stream_handle(stream)))
        return {name: getattr(r, name) for name, _ in _abi.TuneReport._fields_}

    def _status(self, st):
        """CIA_ERR_FALLBACK is informational: the results are valid and the
        check report says what happened; every other error raises."""
        if st == 6:
            self.last_fallback = load().cia_last_error().decode(errors="replace")
            return
        _abi.check(st)

    # ------------------------------------------------------------ learned basis (Cucker--Smale)
    def set_basis(self, basis: "Basis"):
        _abi.check(self._lib.cia_plan_set_basis(self._h, basis._h))

    def sample_pairs(self, count, seed=0, out=None, stream=None):
        """Training pairs [count, 5] drawn from the resident state."""
        import torch
        if out is None:
            out = torch.empty((int(count), 5), dtype=torch.float32, device="cuda")
        _abi.check(self._lib.cia_plan_sample_pairs(self._h, int(count), int(seed),
                                                   _dev_ptr(out, "float32", 5 * int(count)),
                                                   _stream_handle(stream)))
        return out

    def set_check(self, every, bound):
        _abi.check(self._lib.cia_plan_set_check(self._h, int(every), float(bound)))

    def check_report(self) -> dict:
        r = _abi.CheckReport()
        _abi.check(self._lib.cia_plan_get_check(self._h, ctypes.byref(r)))
        return {name: getattr(r, name) for name, _ in _abi.CheckReport._fields_}

    def learn_fit(self, basis: "Basis", x0, *, dt, steps, snapshots, pairs, seed=0,
                  batch=16384, epochs=1, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                  lr_final=0.0, stream=None) -> dict:
        o = _abi.LearnOptions(float(dt), int(steps), int(snapshots), int(pairs), int(seed),
                              _abi.FitOptions(int(batch), int(epochs),
                                              _abi.AdamOptions(lr, beta1, beta2, eps),
                                              float(lr_final)))
        rep = _abi.LearnReport()
        _abi.check(self._lib.cia_learn_fit(self._h, basis._h, _dev_ptr(x0, "float64", self.size),
                                           ctypes.byref(o), ctypes.byref(rep),
                                           _stream_handle(stream)))
        return {"pairs": rep.pairs, "steps": rep.fit.steps, "first_loss": rep.fit.first_loss,
                "last_epoch_loss": rep.fit.last_epoch_loss}

    def profile_begin(self, capacity: int):
        _abi.check(self._lib.cia_profile_begin(self._h, int(capacity)))

    def profile_end(self) -> dict:
        pr = _abi.Profile()
        _abi.check(self._lib.cia_profile_end(self._h, ctypes.byref(pr)))
        return {"stage_launches": pr.stage_launches, "stage_ms": pr.stage_ms,
                "other_launches": pr.other_launches}

    def sync(self, stream=None):
        _abi.check(self._lib.cia_sync(self._h, _stream_handle(stream)))

    def selftest_bounded_wait(self, limit_ns=1_000_000, stream=None):
        """Launch a kernel whose bounded wait must give up (failure detection)."""
        _abi.check(self._lib.cia_selftest_bounded_wait(self._h, int(limit_ns), _stream_handle(stream)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cia_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Basis:
    """Learned separable basis phi of the Cucker--Smale weight (include/cia_basis.h).

    params: host float32 vector of CIA_BASIS_PARAMS entries packed as
    W1 [128, 2], b1 [128], W2 [64, 128], b2 [64].
    """

    PARAMS = _abi.CIA_BASIS_PARAMS
    HIDDEN = _abi.CIA_BASIS_HIDDEN
    RANK = _abi.CIA_BASIS_RANK

    def __init__(self, params):
        lib = load()
        self._lib = lib
        params = np.ascontiguousarray(params, dtype=np.float32)
        if params.shape != (self.PARAMS,):
            raise ValueError("params must have %d entries" % self.PARAMS)
        handle = ctypes.c_void_p()
        _abi.check(lib.cia_basis_create(params.ctypes.data, ctypes.byref(handle)))
        self._h = handle

    @classmethod
    def params_fourier(cls, K, sigma, beta, L, seed=0) -> np.ndarray:
        """Parameters that make phi the rank-64 Fourier basis of the weight on [-L, L]^2."""
        out = np.empty(cls.PARAMS, dtype=np.float32)
        _abi.check(load().cia_basis_params_fourier(float(K), float(sigma), float(beta), float(L),
                                                   int(seed), out.ctypes.data))
        return out

    def params(self) -> np.ndarray:
        out = np.empty(self.PARAMS, dtype=np.float32)
        _abi.check(self._lib.cia_basis_get_params(self._h, out.ctypes.data))
        return out

    def features(self, x, out=None, stream=None):
        """phi(x) for x (CUDA float32, [B, 2]); returns [B, 64] float32."""
        import torch
        B = x.shape[0]
        if out is None:
            out = torch.empty((B, self.RANK), dtype=torch.float32, device=x.device)
        _abi.check(self._lib.cia_basis_features(self._h, _dev_ptr(x, "float32", 2 * B), B,
                                                _dev_ptr(out, "float32", self.RANK * B),
                                                _stream_handle(stream)))
        return out

    def pair_grad(self, pairs, grad=None, loss=None, stream=None):
        """Gradient of the mean squared pair loss over pairs (CUDA float32, [B, 5])."""
        import torch
        B = pairs.shape[0]
        if grad is None:
            grad = torch.empty(self.PARAMS, dtype=torch.float32, device=pairs.device)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float64, device=pairs.device)
        _abi.check(self._lib.cia_basis_pair_grad(self._h, _dev_ptr(pairs, "float32", 5 * B), B,
                                                 _dev_ptr(grad, "float32", self.PARAMS),
                                                 _dev_ptr(loss, "float64", 1),
                                                 _stream_handle(stream)))
        return grad, loss

    def adam_step(self, grad, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        o = _abi.AdamOptions(lr, beta1, beta2, eps)
        _abi.check(self._lib.cia_basis_adam_step(self._h, _dev_ptr(grad, "float32", self.PARAMS),
                                                 ctypes.byref(o), _stream_handle(stream)))

    def fit(self, pairs, batch=16384, epochs=1, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
            lr_final=0.0, stream=None) -> dict:
        B = pairs.shape[0]
        o = _abi.FitOptions(int(batch), int(epochs), _abi.AdamOptions(lr, beta1, beta2, eps),
                            float(lr_final))
        rep = _abi.FitReport()
        _abi.check(self._lib.cia_basis_fit(self._h, _dev_ptr(pairs, "float32", 5 * B), B,
                                           ctypes.byref(o), ctypes.byref(rep),
                                           _stream_handle(stream)))
        return {"steps": rep.steps, "first_loss": rep.first_loss,
                "last_epoch_loss": rep.last_epoch_loss}

    def sync(self, stream=None):
        _abi.check(self._lib.cia_basis_sync(self._h, _stream_handle(stream)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cia_basis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
