"""Learned penumbra surrogate: state, training data, training, checkpoints.

Not in the paper: this library's estimate of the Listing 5 (RSMSS) answer of
an edge fragment from its 5x5 shadow-test pattern, in-texel offsets and depth
gap (include/rbsm.h, "Learned penumbra surrogate").  Every step runs in the
library's kernels (rbsm_mlp_*): the training data come from the exact walk,
the gradient and the Adam update from the tensor-core training kernels.
This module only moves buffers and loops over steps.
"""
import ctypes
import json
import os

import numpy as np
import torch

from . import _native as N
from .api import _stream_handle, frags_desc, map_desc, _params

SAMPLE_BYTES = ctypes.sizeof(N.rbsm_sample)    # 20
N_PARAMS = N.RBSM_MLP_PARAMS
CHECKPOINT_MAGIC = "rbsm-surrogate-v1"


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Surrogate:
    """A network state block on one device, loaded from float32 parameters
    (the canonical vector order W1, b1, W2, b2, W3, b3; see include/rbsm.h)."""

    def __init__(self, params, device="cuda"):
        nbytes = N.lib().rbsm_mlp_state_bytes()
        self.device = torch.device(device)
        # 256-byte aligned: the caching allocator aligns blocks to 512 bytes
        self.state = torch.zeros(nbytes // 4 + 64, dtype=torch.float32, device=self.device)
        self.step = 0
        self.load(params)

    @staticmethod
    def flatten(p):
        """Canonical float32 vector from a dict of W1, b1, W2, b2, W3, b3."""
        return np.concatenate([np.asarray(p[k], np.float32).reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])

    @staticmethod
    def unflatten(v):
        v = np.asarray(v, np.float64)
        shapes = [("W1", (32, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 2)), ("b3", (2,))]
        out, o = {}, 0
        for k, sh in shapes:
            n = int(np.prod(sh))
            out[k] = v[o:o + n].reshape(sh)
            o += n
        assert o == N_PARAMS
        return out

    def load(self, params):
        vec = params if isinstance(params, np.ndarray) and params.ndim == 1 else self.flatten(params)
        vec = np.ascontiguousarray(vec, np.float32)
        if vec.shape != (N_PARAMS,):
            raise ValueError("expected %d parameters" % N_PARAMS)
        self.step = 0
        self.trust = None
        self._host = torch.from_numpy(vec.copy()).pin_memory()
        N.check("rbsm_mlp_load", N.lib().rbsm_mlp_load(_ptr(self.state), _ptr(self._host), _stream_handle(None)))
        torch.cuda.current_stream().synchronize()

    def set_trust(self, bitmap):
        """Trusted-pattern bitmap (uint32 array of RBSM_MLP_TRUST_WORDS words;
        bit p & 31 of word p >> 5 for pattern p), or None for none."""
        if bitmap is None:
            self.trust = None
            N.check("rbsm_mlp_set_trust", N.lib().rbsm_mlp_set_trust(_ptr(self.state), None, _stream_handle(None)))
        else:
            bitmap = np.ascontiguousarray(bitmap, np.uint32)
            if bitmap.shape != (N.RBSM_MLP_TRUST_WORDS,):
                raise ValueError("expected %d words" % N.RBSM_MLP_TRUST_WORDS)
            self.trust = bitmap
            host = torch.from_numpy(bitmap.view(np.int32)).pin_memory()
            N.check("rbsm_mlp_set_trust", N.lib().rbsm_mlp_set_trust(_ptr(self.state), _ptr(host),
                                                                     _stream_handle(None)))
        torch.cuda.current_stream().synchronize()

    @staticmethod
    def trust_bitmap(patterns):
        """Bitmap with the bits of the given 25-bit patterns set."""
        p = np.unique(np.asarray(patterns, np.uint32))
        words = np.zeros(N.RBSM_MLP_TRUST_WORDS, np.uint32)
        np.bitwise_or.at(words, p >> 5, np.left_shift(np.uint32(1), p & np.uint32(31)))
        return words

    def params(self):
        out = torch.empty(N_PARAMS, dtype=torch.float32, pin_memory=True)
        N.check("rbsm_mlp_store", N.lib().rbsm_mlp_store(_ptr(self.state), _ptr(out), _stream_handle(None)))
        torch.cuda.current_stream().synchronize()
        return out.numpy().copy()

    # --------------------------------------------------------------- data --
    @staticmethod
    def dataset(maps_frags, capacity, max_dist=N.RBSM_MAXDIST_DEFAULT, device="cuda", in_window=False):
        """Training samples (a uint8 tensor of capacity x 20 bytes) from every
        edge fragment of the given (depth, x, y, z) CUDA tensors (with
        in_window, only those whose walks stop inside the 5x5 window), until
        `capacity`; returns (samples, count)."""
        samples = torch.empty(capacity * SAMPLE_BYTES, dtype=torch.uint8, device=device)
        counter = torch.zeros(1, dtype=torch.int64, device=device)
        for depth, x, y, z in maps_frags:
            m, f, p = map_desc(depth), frags_desc(x, y, z), _params(max_dist)
            p.flags = N.RBSM_DATASET_IN_WINDOW if in_window else 0
            N.check("rbsm_mlp_dataset",
                    N.lib().rbsm_mlp_dataset(ctypes.byref(m), ctypes.byref(f), ctypes.byref(p), _ptr(samples),
                                             capacity, _ptr(counter), _stream_handle(None)))
        count = min(int(counter.item()), capacity)
        return samples, count

    @staticmethod
    def unpack(samples, count):
        """Host numpy view of packed samples: dict of bits, fx, fy, gap, label."""
        raw = samples[:count * SAMPLE_BYTES].cpu().numpy()
        rec = raw.view(np.dtype([("bits", "<u4"), ("fx", "<f4"), ("fy", "<f4"), ("gap", "<f4"), ("label", "<f4")]))
        return {k: rec[k].copy() for k in ("bits", "fx", "fy", "gap", "label")}

    @staticmethod
    def pack(feat, labels, device="cuda"):
        """Packed samples from host arrays (bits, fx, fy, gap) and labels."""
        n = len(labels)
        rec = np.empty(n, np.dtype([("bits", "<u4"), ("fx", "<f4"), ("fy", "<f4"), ("gap", "<f4"), ("label", "<f4")]))
        for k in ("bits", "fx", "fy", "gap"):
            rec[k] = feat[k]
        rec["label"] = labels
        return torch.from_numpy(rec.view(np.uint8).copy()).to(device), n

    # -------------------------------------------------------- training --
    def grad(self, samples, order):
        """Accumulate the gradient of one minibatch (order: int32 CUDA tensor)."""
        N.check("rbsm_mlp_grad", N.lib().rbsm_mlp_grad(_ptr(self.state), _ptr(samples), _ptr(order),
                                                       int(order.numel()), _stream_handle(None)))

    def adam(self, lr):
        self.step += 1
        N.check("rbsm_mlp_adam", N.lib().rbsm_mlp_adam(_ptr(self.state), self.step, float(lr), _stream_handle(None)))

    def train_step(self, samples, order, lr):
        """Gradient of one minibatch and the Adam step, in two kernels."""
        self.step += 1
        N.check("rbsm_mlp_step", N.lib().rbsm_mlp_step(_ptr(self.state), _ptr(samples), _ptr(order),
                                                       int(order.numel()), self.step, float(lr),
                                                       _stream_handle(None)))

    def read_grad(self):
        g = torch.empty(N_PARAMS, dtype=torch.float32, pin_memory=True)
        N.check("rbsm_mlp_read", N.lib().rbsm_mlp_read(_ptr(self.state), _ptr(g), None, _stream_handle(None)))
        return g.numpy().copy()

    def take_loss(self):
        """Loss sum accumulated since the last call (and reset it)."""
        l = torch.zeros(1, dtype=torch.float32, pin_memory=True)
        N.check("rbsm_mlp_read", N.lib().rbsm_mlp_read(_ptr(self.state), None, _ptr(l), _stream_handle(None)))
        N.check("rbsm_mlp_reset_loss", N.lib().rbsm_mlp_reset_loss(_ptr(self.state), _stream_handle(None)))
        return float(l.item())

    def train(self, samples, count, epochs=2, batch=8192, lr=2e-3, seed=0, lr_decay=0.5, log=None):
        """Adam over shuffled minibatches of the first `count` samples.
        Returns the mean training loss of every epoch."""
        rng = np.random.Generator(np.random.PCG64(9000 + seed))
        history = []
        steps_per_epoch = max(1, count // batch)
        for ep in range(epochs):
            perm = torch.from_numpy(rng.permutation(count).astype(np.int32)).to(self.device)
            self.take_loss()
            for s in range(steps_per_epoch):
                self.train_step(samples, perm[s * batch:(s + 1) * batch], lr)
            history.append(self.take_loss() / (steps_per_epoch * batch))
            if log:
                log("epoch %d loss %.6f lr %.2e" % (ep, history[-1], lr))
            lr *= lr_decay
        return history

    def forward(self, samples, count):
        out = torch.empty(count * 2, dtype=torch.float32, device=self.device)
        N.check("rbsm_mlp_forward", N.lib().rbsm_mlp_forward(_ptr(self.state), _ptr(samples), int(count), _ptr(out),
                                                             _stream_handle(None)))
        return out.view(count, 2)

    # ------------------------------------------------------ checkpoints --
    def save(self, path, meta=None):
        """Parameters (float32) plus a header: dims, Adam step, caller's meta."""
        header = {"magic": CHECKPOINT_MAGIC, "dims": [32, 64, 64, 2], "params": N_PARAMS, "step": self.step}
        header.update(meta or {})
        extra = {} if self.trust is None else {"trust": self.trust}
        np.savez_compressed(path, params=self.params(), header=np.array(json.dumps(header)), **extra)

    @classmethod
    def from_checkpoint(cls, path, device="cuda"):
        z = np.load(path)
        header = json.loads(str(z["header"]))
        if header.get("magic") != CHECKPOINT_MAGIC or int(header.get("params", 0)) != N_PARAMS:
            raise ValueError("%s is not a surrogate checkpoint of this library" % path)
        s = cls(z["params"], device=device)
        s.step = int(header.get("step", 0))
        s.header = header
        if "trust" in z.files:
            s.set_trust(z["trust"])
        return s
