"""Learned control proposal: the network context (thin binding of the
kp_mlp_* entry points) and its training pipeline.

The network maps 24 node features (zero padded to 32) through two ReLU
layers of 256 units to a Gaussian over 4 normalised quantities (3 controls
and the duration).  Inference and training run in the library's BF16
tensor-core kernels; this module only marshals arguments and drives the
harvest -> train -> use loop.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .planner import KpError, OK, lib

N_IN, N_H, N_OUT = 32, 256, 8


def num_params() -> int:
    return lib().kp_mlp_num_params()


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform hidden layers, small output layer, zero biases (log-std
    bias 0: unit standard deviation in normalised units)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_out, fan_in, gain in ((N_H, N_IN, 1.0), (N_H, N_H, 1.0), (N_OUT, N_H, 0.1)):
        a = gain * np.sqrt(6.0 / fan_in)
        parts += [rng.uniform(-a, a, fan_out * fan_in), np.zeros(fan_out)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == num_params()
    return p


def split(p):
    """(W1, b1, W2, b2, W3, b3) views of a flat parameter vector."""
    sizes = [(N_H, N_IN), (N_H,), (N_H, N_H), (N_H,), (N_OUT, N_H), (N_OUT,)]
    out, o = [], 0
    for s in sizes:
        n = int(np.prod(s))
        out.append(p[o:o + n].reshape(s))
        o += n
    return out


class Mlp:
    """One network context in a device arena (torch uint8 tensor)."""

    def __init__(self, params=None, max_batch=4096, device=None, stream=None, seed=0):
        import torch
        L = lib()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        p = np.ascontiguousarray(init_params(seed) if params is None else params, np.float32)
        nbytes = L.kp_mlp_required_bytes(int(max_batch))
        self.arena = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.max_batch = int(max_batch)
        self._ctx = C.c_void_p()
        st = L.kp_mlp_create(C.c_void_p(self.arena.data_ptr()), int(nbytes), int(max_batch),
                             p.ctypes.data_as(C.POINTER(C.c_float)),
                             C.c_void_p(self.stream.cuda_stream), C.byref(self._ctx))
        if st != OK:
            raise KpError(st, "kp_mlp_create failed")

    def close(self):
        if getattr(self, "_ctx", None):
            lib().kp_mlp_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _chk(st, what):
        if st != OK:
            raise KpError(st, what)

    def params(self) -> np.ndarray:
        out = np.zeros(num_params(), np.float32)
        self._chk(lib().kp_mlp_get_params(self._ctx, out.ctypes.data_as(C.POINTER(C.c_float))),
                  "kp_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        self._chk(lib().kp_mlp_set_params(self._ctx, p.ctypes.data_as(C.POINTER(C.c_float))),
                  "kp_mlp_set_params")

    def forward(self, x):
        """x: CUDA float32 [M, 32] -> CUDA float32 [M, 8] (mean[4], log_std[4])."""
        import torch
        x = x.contiguous()
        out = torch.empty((x.shape[0], N_OUT), dtype=torch.float32, device=x.device)
        self._chk(lib().kp_mlp_forward(self._ctx, x.data_ptr(), x.shape[0], out.data_ptr()),
                  "kp_mlp_forward")
        return out

    def gradients(self, x, t):
        g = np.zeros(num_params(), np.float32)
        loss = C.c_float()
        self._chk(lib().kp_mlp_gradients(self._ctx, x.contiguous().data_ptr(),
                                         t.contiguous().data_ptr(), x.shape[0],
                                         g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)),
                  "kp_mlp_gradients")
        return g, loss.value

    def train_epoch(self, x, t, perm, lr=1e-3):
        """One epoch over rows perm of (x, t) in mini-batches of max_batch
        rows, driven on the device; returns the mean mini-batch loss."""
        import torch
        perm = perm.to(device=x.device, dtype=torch.int32).contiguous()
        loss = C.c_float()
        self._chk(lib().kp_mlp_train_epoch(self._ctx, x.contiguous().data_ptr(),
                                           t.contiguous().data_ptr(), perm.data_ptr(),
                                           int(perm.shape[0]), float(lr), C.byref(loss)),
                  "kp_mlp_train_epoch")
        return loss.value

    def train_step(self, x, t, lr=1e-3, want_loss=False):
        loss = C.c_float()
        self._chk(lib().kp_mlp_train_step(self._ctx, x.data_ptr(), t.data_ptr(), x.shape[0],
                                          float(lr), C.byref(loss) if want_loss else None),
                  "kp_mlp_train_step")
        return loss.value if want_loss else None


def harvest(make_workload, seeds, n_pairs, max_iters=400, planner=None, per_query_cap=1 << 18,
            seed=0):
    """Plain planner runs on the given layouts; from each, an even share of
    n_pairs training pairs (parent features -> draw of a sample that reached
    a new sub-region), chosen uniformly at random (seeded) among all the
    pairs that query produced, so that every layout and every stage of its
    search is represented.  Returns CUDA tensors (features [n, 32], targets
    [n, 4]) of at most n_pairs rows."""
    import torch
    from .planner import Planner
    w0 = make_workload(seeds[0])
    pl = planner or Planner(w0)
    pl.set_harvest(per_query_cap)
    share = -(-n_pairs // len(seeds))  # ceil
    rng = np.random.Generator(np.random.PCG64(seed))
    feats, targs, have = [], [], 0
    for s in seeds:
        w = make_workload(s)
        pl.set_obstacles(w.boxes)
        pl.w = w
        pl.harvest_reset()
        pl.plan(max_iters=max_iters, x_init=w.x_init)
        f, t = pl.harvest()
        take = min(len(f), share, n_pairs - have)
        if take <= 0:
            continue
        idx = torch.from_numpy(np.sort(rng.choice(len(f), size=take, replace=False))).to(f.device)
        feats.append(f.index_select(0, idx).clone())
        targs.append(t.index_select(0, idx).clone())
        have += take
        if have >= n_pairs:
            break
    pl.set_harvest(0)
    return torch.cat(feats), torch.cat(targs)


def train(mlp, feats, targs, epochs=3, batch=4096, lr=1e-3, seed=0, log_every=0):
    """Mini-batch Adam on the Gaussian negative log-likelihood; returns the
    per-epoch mean losses."""
    import torch
    n = feats.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for ep in range(epochs):
        # drawn as int32 on the host: only a copy reaches the device
        perm = torch.randperm(n, generator=g, dtype=torch.int32).to(feats.device)
        if batch == mlp.max_batch:
            hist.append(mlp.train_epoch(feats, targs, perm, lr))
            continue
        losses = []
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            x = feats.index_select(0, idx).contiguous()
            t = targs.index_select(0, idx).contiguous()
            want = (i // batch) % 16 == 0
            loss = mlp.train_step(x, t, lr, want_loss=want)
            if want:
                losses.append(loss)
        hist.append(float(np.mean(losses)) if losses else float("nan"))
    return hist
