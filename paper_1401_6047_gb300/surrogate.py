"""Python binding of the surrogate ABI in ``include/bte_surrogate.h`` (ctypes,
argument marshalling only; every computation runs in the CUDA library).

``Surrogate.fit`` draws the per-member minibatch orders with numpy (seeded)
and passes them, with the learning-rate schedule, to ``bte_sur_train``;
initial weights come from the caller (``init_params``) through
``bte_sur_set_params``, so the library itself draws no random numbers.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import bte
from . import workloads as W

N_IN, N_OUT = 5, 2


class bte_sur_config(ctypes.Structure):
    _fields_ = [("members", ctypes.c_int32), ("width", ctypes.c_int32),
                ("batch_capacity", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("x_lo", ctypes.c_double * 5), ("x_hi", ctypes.c_double * 5),
                ("y_mean", ctypes.c_double * 2), ("y_std", ctypes.c_double * 2),
                ("stream", ctypes.c_void_p)]


_sig_done = False


def _lib():
    global _sig_done
    L = bte.lib()
    if not _sig_done:
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        fp = ctypes.POINTER(ctypes.c_float)
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        sig = {
            "bte_sur_create": ([ctypes.POINTER(bte_sur_config), ctypes.POINTER(vp)], ctypes.c_int),
            "bte_sur_param_count": ([vp], i64),
            "bte_sur_set_params": ([vp, fp], ctypes.c_int),
            "bte_sur_get_params": ([vp, fp], ctypes.c_int),
            "bte_sur_set_data": ([vp, fp, fp, i64], ctypes.c_int),
            "bte_sur_train": ([vp, i32p, i32, i32, fp, dp], ctypes.c_int),
            "bte_sur_grad": ([vp, fp, fp, i32, fp, dp], ctypes.c_int),
            "bte_sur_predict": ([vp, fp, i64, fp, fp, u8p, ctypes.c_double], ctypes.c_int),
            "bte_sur_predict_device": ([vp, vp, i64, vp, vp, vp, ctypes.c_double], ctypes.c_int),
            "bte_sur_protocol": ([dp, i32, ctypes.POINTER(bte.bte_params)], ctypes.c_int),
            "bte_sur_hybrid": ([vp, dp, i64, ctypes.c_double, i32,
                                ctypes.POINTER(bte.bte_batch_opts), dp, u8p, i32p], ctypes.c_int),
            "bte_sur_destroy": ([vp], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _sig_done = True
    return L


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        assert a.shape == shape, (a.shape, shape)
    return a


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def box_bounds():
    lo = np.array([v[0] for v in W.SWEEP_BOX.values()])
    hi = np.array([v[1] for v in W.SWEEP_BOX.values()])
    return lo, hi


def protocol(x, precision: int = W.FP32_MIXED) -> bte.bte_params:
    """Solver parameters the library assigns to surrogate point x."""
    xx = np.ascontiguousarray(x, dtype=np.float64)
    out = bte.bte_params()
    bte._check(_lib().bte_sur_protocol(_p(xx, ctypes.c_double), int(precision), ctypes.byref(out)))
    return out


def init_params(members: int, seed: int = 0, width: int = 256) -> np.ndarray:
    """Seeded initial weights [members][count]: W ~ U(-sqrt(3/fan_in),
    sqrt(3/fan_in)), biases 0; member m uses seed + m."""
    out = []
    for m in range(members):
        rng = np.random.default_rng(seed + m)
        parts = []
        for name, shp in (("W1", (width, 5)), ("b1", (width,)), ("W2", (width, width)),
                          ("b2", (width,)), ("W3", (width, width)), ("b3", (width,)),
                          ("W4", (2, width)), ("b4", (2,))):
            if name.startswith("W"):
                lim = math.sqrt(3.0 / shp[1])
                parts.append(rng.uniform(-lim, lim, size=shp).ravel())
            else:
                parts.append(np.zeros(int(np.prod(shp))))
        out.append(np.concatenate(parts))
    return np.stack(out).astype(np.float32)


class Surrogate:
    """Ensemble of MLPs on the GPU (a ``bte_sur`` handle)."""

    def __init__(self, y_mean, y_std, members: int = 8, batch_capacity: int = 16384,
                 x_lo=None, x_hi=None, stream: int = 0):
        self._lib = _lib()
        lo, hi = box_bounds()
        cfg = bte_sur_config()
        cfg.members, cfg.width, cfg.batch_capacity, cfg.reserved = members, 256, batch_capacity, 0
        cfg.x_lo[:] = list(lo if x_lo is None else x_lo)
        cfg.x_hi[:] = list(hi if x_hi is None else x_hi)
        cfg.y_mean[:] = [float(v) for v in y_mean]
        cfg.y_std[:] = [float(v) for v in y_std]
        cfg.stream = ctypes.c_void_p(stream or None)
        self.cfg = cfg
        self.members = members
        self.capacity = batch_capacity
        self._h = ctypes.c_void_p()
        bte._check(self._lib.bte_sur_create(ctypes.byref(cfg), ctypes.byref(self._h)))
        self.count = int(self._lib.bte_sur_param_count(self._h))

    def close(self):
        if self._h:
            self._lib.bte_sur_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, p) -> None:
        p = _f32(p, (self.members, self.count))
        bte._check(self._lib.bte_sur_set_params(self._h, _p(p, ctypes.c_float)))

    def get_params(self) -> np.ndarray:
        p = np.zeros((self.members, self.count), dtype=np.float32)
        bte._check(self._lib.bte_sur_get_params(self._h, _p(p, ctypes.c_float)))
        return p

    def set_data(self, x, y) -> None:
        x = _f32(x)
        y = _f32(y)
        assert x.ndim == 2 and x.shape[1] == N_IN and y.shape == (x.shape[0], N_OUT)
        self.n_data = x.shape[0]
        bte._check(self._lib.bte_sur_set_data(self._h, _p(x, ctypes.c_float), _p(y, ctypes.c_float),
                                              x.shape[0]))

    def train(self, order, lr, return_loss: bool = True):
        order = np.ascontiguousarray(order, dtype=np.int32)
        steps, members, batch = order.shape
        assert members == self.members
        lr = _f32(lr, (steps,))
        loss = np.zeros((steps, members)) if return_loss else None
        bte._check(self._lib.bte_sur_train(self._h, _p(order, ctypes.c_int32), steps, batch,
                                           _p(lr, ctypes.c_float),
                                           _p(loss, ctypes.c_double) if return_loss else None))
        return loss

    def fit(self, x, y, epochs: int, batch: int = 1024, lr: float = 2e-3, lr_min: float = 2e-5,
            seed: int = 0, log=None):
        """Adam with a cosine learning-rate decay over all steps; member m
        shuffles with seed (seed, m, epoch).  Returns the mean loss per epoch."""
        self.set_data(x, y)
        n = self.n_data
        steps_per = n // batch
        total = epochs * steps_per
        hist = []
        for ep in range(epochs):
            order = np.empty((steps_per, self.members, batch), dtype=np.int32)
            for m in range(self.members):
                perm = np.random.default_rng([seed, m, ep]).permutation(n)[: steps_per * batch]
                order[:, m, :] = perm.reshape(steps_per, batch)
            s0 = ep * steps_per
            t = (np.arange(s0, s0 + steps_per) + 0.5) / total
            lrs = lr_min + 0.5 * (lr - lr_min) * (1 + np.cos(np.pi * t))
            loss = self.train(order, lrs)
            hist.append(float(loss.mean()))
            if log:
                log(ep, hist[-1])
        return hist

    def grad(self, x, t):
        x = _f32(x)
        t = _f32(t)
        n = x.shape[0]
        g = np.zeros((self.members, self.count), dtype=np.float32)
        loss = np.zeros(self.members)
        bte._check(self._lib.bte_sur_grad(self._h, _p(x, ctypes.c_float), _p(t, ctypes.c_float), n,
                                          _p(g, ctypes.c_float), _p(loss, ctypes.c_double)))
        return loss, g

    def predict(self, x, threshold: float = 1e-3, out=None):
        """(mean [n, 2], std [n, 2], mask [n] bool) of host inputs x [n, 5].
        `out` = (mean float32 [n, 2], std float32 [n, 2], mask uint8 [n]) host
        arrays to fill instead (page-locked ones let the copies overlap the
        inference); the mask is then returned as the uint8 array itself."""
        x = _f32(x)
        n = x.shape[0]
        if out is None:
            mean = np.zeros((n, 2), dtype=np.float32)
            std = np.zeros((n, 2), dtype=np.float32)
            mask = np.zeros(n, dtype=np.uint8)
        else:
            mean, std, mask = out
            for a, shp, dt in ((mean, (n, 2), np.float32), (std, (n, 2), np.float32),
                               (mask, (n,), np.uint8)):
                if a.shape != shp or a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("out arrays must be C-contiguous float32 [n, 2] x 2 and uint8 [n]")
        bte._check(self._lib.bte_sur_predict(self._h, _p(x, ctypes.c_float), n, _p(mean, ctypes.c_float),
                                             _p(std, ctypes.c_float), _p(mask, ctypes.c_uint8),
                                             float(threshold)))
        return (mean, std, mask.astype(bool)) if out is None else (mean, std, mask)

    def predict_device(self, x_ptr: int, n: int, mean_ptr: int, std_ptr: int, mask_ptr: int = 0,
                       threshold: float = 1e-3) -> None:
        bte._check(self._lib.bte_sur_predict_device(self._h, ctypes.c_void_p(x_ptr), int(n),
                                                    ctypes.c_void_p(mean_ptr), ctypes.c_void_p(std_ptr),
                                                    ctypes.c_void_p(mask_ptr or None), float(threshold)))

    def hybrid(self, x, threshold: float = 1e-3, precision: int = W.FP32_MIXED, check: bool = True,
               **batch_opts):
        """(y [n, 2], solved [n] bool, status [n]): surrogate where the
        members agree within threshold, the batched solver elsewhere."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        n = x.shape[0]
        y = np.zeros((n, 2))
        solved = np.zeros(n, dtype=np.uint8)
        status = np.zeros(n, dtype=np.int32)
        o = bte.bte_batch_opts()
        for k in ("tile_m", "chunk_n", "vec", "graph_steps", "max_batch", "max_batch_bytes",
                  "resident", "resident_smem", "walk"):
            setattr(o, k, int(batch_opts.get(k, 0)))
        o.stream = None
        rc = self._lib.bte_sur_hybrid(self._h, _p(x, ctypes.c_double), n, float(threshold),
                                      int(precision), ctypes.byref(o), _p(y, ctypes.c_double),
                                      _p(solved, ctypes.c_uint8), _p(status, ctypes.c_int32))
        if check or rc in (bte.EINVAL, bte.ENOMEM, bte.ECUDA):
            bte._check(rc)
        return y, solved.astype(bool), status
