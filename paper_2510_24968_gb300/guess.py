"""Learned initial density: orchestration over the C-ABI (libfsim).

Every numeric step runs in the library: features and pair-local frames
(fsim_guess_features / fsim_guess_targets), the network's forward, backward and
Adam (fsim_mlp_*), the rotation and assembly of predicted blocks
(fsim_guess_assemble), the converged training densities (fsim_scf), and the
trace/idempotency check with core-Hamiltonian fallback (fsim_scf with a
supplied guess).  This module only moves arrays, draws the seeded initial
weights and minibatch order, and sets the learning-rate schedule (Adam,
lr 1e-3 with cosine decay, as specified for the learned guess).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from fsim_synth import SplitMix64

from .fsim import (FSIM_MIXED, Basis, _check, load)

NFEAT = 48
NOUT = 225
WIDTH = 256


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def layout(basis: Basis):
    n, f, o = C.c_int(), C.c_int(), C.c_int()
    _check(load().fsim_guess_layout(basis.h, C.byref(n), C.byref(f), C.byref(o)))
    return n.value, f.value, o.value


def features(basis: Basis) -> np.ndarray:
    n, f, _ = layout(basis)
    out = np.zeros((n, f), dtype=np.float32)
    _check(load().fsim_guess_features(basis.h, _fp(out)))
    return out


def targets(basis: Basis, D: np.ndarray):
    n, _, o = layout(basis)
    t = np.zeros((n, o), dtype=np.float32)
    m = np.zeros((n, o), dtype=np.float32)
    D = np.ascontiguousarray(D, dtype=np.float64)
    _check(load().fsim_guess_targets(basis.h, D.ctypes.data_as(C.POINTER(C.c_double)), _fp(t), _fp(m)))
    return t, m


def init_params(nin: int, width: int, nout: int, seed: int) -> np.ndarray:
    """Seeded initial weights: normal(0, 1/fan_in) weights, zero biases."""
    rng = SplitMix64(seed)
    parts = []
    for fi, fo in ((nin, width), (width, width), (width, nout)):
        parts.append(np.array([rng.normal() for _ in range(fi * fo)], dtype=np.float32) / math.sqrt(fi))
        parts.append(np.zeros(fo, dtype=np.float32))
    return np.concatenate(parts)


class GuessNet:
    """fsim_mlp handle (device parameters, BF16 tensor-core GEMMs)."""

    def __init__(self, nin=NFEAT, width=WIDTH, nout=NOUT, seed=7, params=None):
        self.nin, self.width, self.nout = nin, width, nout
        p = init_params(nin, width, nout, seed) if params is None else np.asarray(params, dtype=np.float32)
        h = C.c_void_p()
        _check(load().fsim_mlp_create(nin, width, nout, _fp(p), C.byref(h)))
        self.h = h
        self.np = load().fsim_mlp_nparams(h)

    def close(self):
        if getattr(self, "h", None):
            load().fsim_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self, path):
        """Weights file for fsim_scf's learned guess (FSIM_GUESS_LEARNED, guess_model)."""
        import os
        _check(load().fsim_mlp_save(self.h, os.fsencode(path)))

    def adam_step(self, grad: np.ndarray, lr: float, stream=0):
        """One Adam step from a supplied gradient (host FP32, nparams values)."""
        g = np.ascontiguousarray(grad, dtype=np.float32)
        _check(load().fsim_mlp_adam_step(self.h, _fp(g), float(lr), C.c_void_p(stream)))

    def params(self) -> np.ndarray:
        out = np.zeros(self.np, dtype=np.float32)
        _check(load().fsim_mlp_params(self.h, _fp(out), None))
        return out

    def forward(self, x_dev, y_dev, batch, bf16=True, stream=0):
        _check(load().fsim_mlp_forward(self.h, C.c_void_p(x_dev), C.c_void_p(y_dev), batch, int(bf16),
                                       C.c_void_p(stream)))

    def grad(self, x_dev, t_dev, m_dev, batch, bf16=False, stream=0):
        loss = C.c_float()
        g = np.zeros(self.np, dtype=np.float32)
        _check(load().fsim_mlp_grad(self.h, C.c_void_p(x_dev), C.c_void_p(t_dev), C.c_void_p(m_dev), batch,
                                    int(bf16), C.byref(loss), _fp(g), C.c_void_p(stream)))
        return loss.value, g

    def train_step(self, x_dev, t_dev, m_dev, batch, lr, stream=0, want_loss=False):
        loss = C.c_float()
        _check(load().fsim_mlp_train_step(self.h, C.c_void_p(x_dev), C.c_void_p(t_dev), C.c_void_p(m_dev), batch,
                                          float(lr), C.byref(loss) if want_loss else None, C.c_void_p(stream)))
        return loss.value if want_loss else None


def training_data(mols, tau=1e-10):
    """Features, targets and masks from converged densities of the library's SCF."""
    X, T, M = [], [], []
    energies = []
    for mol in mols:
        b = Basis(mol)
        r = b.scf(precision=FSIM_MIXED, tau=tau, want_density=True)
        if not r["converged"]:
            continue
        X.append(features(b))
        t, m = targets(b, r["D"])
        T.append(t)
        M.append(m)
        energies.append(r["e_total"])
    return np.concatenate(X), np.concatenate(T), np.concatenate(M), energies


def training_data_batched(mols, tau=1e-10, chunk=256):
    """training_data() through the library's batched lockstep SCF (mixed
    precision, no FP64 reset: the targets are FP32 blocks), chunk molecules
    per batch; molecules that do not converge are left out."""
    from .fsim import scf_batched
    X, T, M = [], [], []
    energies = []
    for c0 in range(0, len(mols), chunk):
        bases = [Basis(m) for m in mols[c0:c0 + chunk]]
        res = scf_batched(bases, precision=FSIM_MIXED, tau=tau, final_fp64=False, want_density=True)
        for b, r in zip(bases, res):
            if not r["converged"]:
                continue
            X.append(features(b))
            t, m = targets(b, r["D"])
            T.append(t)
            M.append(m)
            energies.append(r["e_total"])
        for b in bases:
            b.close()
    return np.concatenate(X), np.concatenate(T), np.concatenate(M), energies


def train(net: GuessNet, X, T, M, steps=2000, batch=4096, lr0=1e-3, seed=11, log_every=0):
    """Adam with cosine decay over `steps` minibatches (device-resident data)."""
    import torch

    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    Td = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(dev)
    Md = torch.from_numpy(np.ascontiguousarray(M, dtype=np.float32)).to(dev)
    n = X.shape[0]
    batch = min(batch, n)
    rng = SplitMix64(seed)
    order = list(range(n))
    pos = n
    xb = torch.empty((batch, X.shape[1]), dtype=torch.float32, device=dev)
    tb = torch.empty((batch, T.shape[1]), dtype=torch.float32, device=dev)
    mb = torch.empty_like(tb)
    losses = []
    for s in range(steps):
        if pos + batch > n:
            rng.shuffle(order)
            perm = torch.tensor(order, device=dev)
            pos = 0
        idx = perm[pos:pos + batch]
        pos += batch
        torch.index_select(Xd, 0, idx, out=xb)
        torch.index_select(Td, 0, idx, out=tb)
        torch.index_select(Md, 0, idx, out=mb)
        lr = lr0 * 0.5 * (1 + math.cos(math.pi * s / steps))
        want = log_every and (s % log_every == 0 or s == steps - 1)
        loss = net.train_step(xb.data_ptr(), tb.data_ptr(), mb.data_ptr(), batch, lr, want_loss=bool(want))
        if want:
            losses.append((s, loss))
    return losses


def combine_gradients(grad: np.ndarray, mask_sum: float) -> np.ndarray:
    """Gradient of the whole minibatch from each rank's share of it.  The loss
    is sum(mask (y - t)^2) / sum(mask) per call, so a share's gradient is
    weighted by its mask sum: g = sum_r w_r g_r / sum_r w_r (one all-reduce of
    the weighted gradient and the weight; the identity on one rank)."""
    import torch
    import torch.distributed as dist
    buf = torch.from_numpy(np.concatenate([np.asarray(grad, dtype=np.float64) * mask_sum, [float(mask_sum)]]))
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if dist.get_backend() == "nccl":
            buf = buf.cuda()
        dist.all_reduce(buf)
        buf = buf.cpu()
    return (buf[:-1] / buf[-1]).numpy().astype(np.float32)


def train_data_parallel(net: GuessNet, X, T, M, steps=2000, batch=4096, lr0=1e-3, seed=11):
    """Data-parallel training: every rank holds the same initial weights and its
    own training shard; per step each rank draws a minibatch of batch/world rows
    from its shard, the gradients are combined over the ranks
    (combine_gradients) and every replica takes the same Adam step, so the
    replicas stay equal.  Cosine learning-rate decay as in train()."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank() if world > 1 else 0
    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    Td = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(dev)
    Md = torch.from_numpy(np.ascontiguousarray(M, dtype=np.float32)).to(dev)
    n = X.shape[0]
    b = max(1, min(batch // world, n))
    rng = SplitMix64(seed + 7919 * rank)
    order = list(range(n))
    pos = n
    losses = []
    for s in range(steps):
        if pos + b > n:
            rng.shuffle(order)
            perm = torch.tensor(order, device=dev)
            pos = 0
        idx = perm[pos:pos + b]
        pos += b
        xb, tb, mb = Xd.index_select(0, idx), Td.index_select(0, idx), Md.index_select(0, idx)
        loss, g = net.grad(xb.data_ptr(), tb.data_ptr(), mb.data_ptr(), b, bf16=True)
        g = combine_gradients(g, float(mb.sum().item()))
        net.adam_step(g, lr0 * 0.5 * (1 + math.cos(math.pi * s / steps)))
        losses.append(loss)
    return losses


def predict_density(basis: Basis, net: GuessNet) -> np.ndarray:
    """Initial density of a molecule from the network (host nbf x nbf)."""
    import torch

    x = torch.from_numpy(features(basis)).cuda()
    y = torch.empty((x.shape[0], NOUT), dtype=torch.float32, device="cuda")
    net.forward(x.data_ptr(), y.data_ptr(), x.shape[0], bf16=True)
    D = torch.zeros((basis.nbf, basis.nbf), dtype=torch.float64, device="cuda")
    _check(load().fsim_guess_assemble(basis.h, C.c_void_p(y.data_ptr()), C.c_void_p(D.data_ptr()), None))
    return D.cpu().numpy()
