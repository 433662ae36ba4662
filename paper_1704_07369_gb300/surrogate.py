"""Training and use of the learned surrogate through the C ABI (argument marshalling only).

The surrogate maps a cell's low Fourier modes of F (|k| <= EF_FEATURE_K) to the same modes of
Q^sigma[F].  Training data are produced by the library itself (ef_collide on seeded BKW-family
cells, then ef_features of F and of Q); the network is trained by the library's tensor-core MLP
kernels (ef_mlp_train_step); inference goes through ef_surrogate_infer, which gates every cell,
audits a seeded fraction against the plain operator and falls back on the device.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (EF_DIAG_STRIDE, EF_FEATURE_STRIDE, EF_KERNEL_HARD_SPHERE, EF_PREC_F32, MLP, Plan, Surrogate,
               ef_features, ef_moments_entropy)
from . import inputs


def make_plan(kernel=EF_KERNEL_HARD_SPHERE, N=32, L=8.0, R=32, prec=EF_PREC_F32):
    return Plan(3, N, L, kernel, R, prec)


def features_of_family(plan, ncells, seed, chunk=2048, device="cuda"):
    """(featF, featQ, mom): features [ncells, EF_FEATURE_STRIDE] of BKW-family cells and of Q^sigma
    of them, and the cells' moments [ncells, EF_DIAG_STRIDE] (FP64)."""
    N, L = plan.N, plan.L
    featF = torch.zeros(ncells, EF_FEATURE_STRIDE, device=device)
    featQ = torch.zeros(ncells, EF_FEATURE_STRIDE, device=device)
    mom = torch.zeros(ncells, EF_DIAG_STRIDE, dtype=torch.float64, device=device)
    F = torch.empty(chunk, N, N, N, device=device)
    Q = torch.empty_like(F)
    for c0 in range(0, ncells, chunk):
        n = min(chunk, ncells - c0)
        inputs.bkw_family_torch(N, L, n, seed + c0, device=device, out=F[:n])
        plan.collide(F, Q, ncells=n)
        ef_features(plan.handle, F, featF[c0:c0 + n], n)
        ef_features(plan.handle, Q, featQ[c0:c0 + n], n)
        ef_moments_entropy(plan.handle, F, None, mom[c0:c0 + n], n)
    torch.cuda.synchronize()
    return featF, featQ, mom


def loss_mask(nfeat_floats, zero_slot, device="cuda"):
    """Weights of the MSE: 1 everywhere except the zero mode (Qh_0 = 0 by mass conservation)."""
    w = torch.ones(nfeat_floats, device=device)
    w[2 * zero_slot:2 * zero_slot + 2] = 0.0
    return w


def zero_slot(K=6):
    slot = 0
    for k0 in range(-K, K + 1):
        for k1 in range(-K, K + 1):
            for k2 in range(0, K + 1):
                if k0 * k0 + k1 * k1 + k2 * k2 > K * K:
                    continue
                if not (k2 > 0 or (k2 == 0 and (k1 > 0 or (k1 == 0 and k0 >= 0)))):
                    continue
                if (k0, k1, k2) == (0, 0, 0):
                    return slot
                slot += 1
    raise ValueError


class Trainer:
    """Fits the normalisation, then trains the MLP with Adam: a short linear warm-up, then a cosine
    learning-rate decay from lr0 to lr1."""

    def __init__(self, plan, nhidden=512, nlayers=4, batch=1024, max_infer_batch=16384, seed=0, moment_features=True):
        self.plan = plan
        self.nf = 2 * 463
        self.batch = batch
        # with moment_features the input also carries the cell's kinetic temperature and its
        # relative entropy to the local Maxwellian (two scalars from the moments)
        nin = self.nf + 2 if moment_features else self.nf
        self.mlp = MLP(nin, nhidden, nlayers, self.nf, max(batch, max_infer_batch), seed=seed)
        self.sur = Surrogate(plan, self.mlp, max_infer_batch)
        self.wmask = loss_mask(self.nf, zero_slot())

    def fit(self, featF, featQ, mom, epochs=20, lr0=1e-3, lr1=1e-5, seed=0, log=None, warmup=0.02):
        """Fits the normalisation on the training set, then trains the surrogate's network.  The
        normalised training set is kept for fit_checker."""
        X = torch.zeros(featF.shape[0], EF_FEATURE_STRIDE, device=featF.device)
        Y = torch.zeros_like(X)
        rw = torch.zeros(featF.shape[0], device=featF.device)
        self.sur.fit_stats(featF, featQ, mom, X, Y, featF.shape[0], rowweight=rw)
        self.sur.normalize(featF, featQ, mom, X, Y, featF.shape[0])
        self._train_set = (X, Y, rw)
        return self._train(self.mlp, epochs, lr0, lr1, seed, log, warmup)

    def _train(self, net, epochs, lr0, lr1, seed, log, warmup):
        X, Y, rw = self._train_set
        n = X.shape[0] // self.batch * self.batch
        loss = torch.zeros(1, device=X.device)
        g = torch.Generator(device="cpu")
        g.manual_seed(seed)
        steps = epochs * (n // self.batch)
        hist = []
        step = 0
        for ep in range(epochs):
            perm = torch.randperm(X.shape[0], generator=g)[:n].to(X.device)
            Xs, Ys, Rs = X[perm], Y[perm], rw[perm]
            tot = torch.zeros(1, device=X.device)
            for b0 in range(0, n, self.batch):
                lr = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * step / max(1, steps)))
                lr *= min(1.0, (step + 1) / max(1.0, warmup * steps))
                net.train_step(Xs[b0:b0 + self.batch], Ys[b0:b0 + self.batch], self.batch, lr, loss,
                               wmask=self.wmask, rowweight=Rs[b0:b0 + self.batch])
                tot += loss
                step += 1
            hist.append(float(tot.item()) / (n // self.batch))
            if log:
                log(ep, hist[-1])
        return hist

    def fit_checker(self, epochs=20, lr0=1e-3, lr1=1e-5, seed=1, init_seed=101, log=None, warmup=0.02):
        """Trains the checker network (same widths, another initialisation and sample order) on the
        training set of fit(); ef_surrogate_set_checker then gates cells on the two networks'
        disagreement (calibrate chooses the threshold)."""
        nin = self.mlp.nin
        self.checker = MLP(nin, self.mlp.nhidden, self.mlp.nlayers, self.nf, self.mlp.max_batch, seed=init_seed)
        return self._train(self.checker, epochs, lr0, lr1, seed, log, warmup)

    def calibrate(self, F, ncells, tol=1e-3, margin=0.8, seed=0, budget=None):
        """Chooses the checker threshold on held-out cells F (resident, ncells a multiple of 64): with
        the checker's scores s_i and the delivered band errors e_i against the plain operator, the
        threshold is margin * min{s_i : e_i > tol} (every miss of the calibration set is flagged,
        with room to spare), or the largest score / margin if nothing misses.  With a budget
        (fraction of cells), the threshold is instead the score quantile that flags that fraction.
        Returns (threshold, fraction of calibration cells flagged, misses, misses left unflagged)."""
        from . import ef_features
        q = torch.zeros(ncells, EF_FEATURE_STRIDE, device=F.device)
        flags = torch.zeros(ncells, dtype=torch.int32, device=F.device)
        score = torch.zeros(ncells, device=F.device)
        self.sur.set_checker(self.checker, 3.0e38)
        self.sur.infer_ex(F, q, flags, ncells, score=score, audit_fraction=0.0, seed=seed, tol=tol)
        Q = torch.empty_like(F)
        self.plan.collide(F, Q, ncells=ncells)
        ref = torch.zeros_like(q)
        ef_features(self.plan.handle, Q, ref, ncells)
        e = band_rel_l2(q, ref)
        sc = score.double()
        miss = e > tol
        if budget is not None:
            thr = float(torch.quantile(sc, 1.0 - float(budget)))
        elif bool(miss.any()):
            thr = float(margin * sc[miss].min())
        else:
            thr = float(sc.max() / margin)
        self.sur.set_checker(self.checker, thr)
        return thr, float((sc > thr).double().mean()), int(miss.sum()), int((miss & (sc <= thr)).sum())

    def predict(self, F, ncells, audit_fraction=0.0, seed=0, tol=1e-3):
        q = torch.zeros(ncells, EF_FEATURE_STRIDE, device=F.device)
        flags = torch.zeros(ncells, dtype=torch.int32, device=F.device)
        self.sur.infer(F, q, flags, ncells, audit_fraction, seed, tol)
        return q, flags


def band_rel_l2(pred, ref, nf=926):
    """Per-cell relative L2 error over the band (FP32 feature rows)."""
    d = (pred[:, :nf] - ref[:, :nf]).double()
    return torch.sqrt((d * d).sum(1) / (ref[:, :nf].double() ** 2).sum(1))
