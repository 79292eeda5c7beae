"""Learned warm start of PCG: generate training pairs with the solver, train
the network of include/lq2d_warmstart.h on the GPU, and solve from its
guess.

Algorithm 1 accepts any initial iterate delta^(0) (r^(0) = r_delta -
Delta delta^(0)) and stops only on the tolerance, so the network can change
how many iterations a solve takes but not what it converges to; a zero
start remains the fallback.  Every arithmetic step (solver, network forward
and backward passes, Adam) runs in the library's CUDA kernels; this module
only moves buffers and loops.
"""
from __future__ import annotations

import time

import numpy as np

from . import lq2d, synth


def _torch():
    import torch
    return torch


class WarmStart:
    """One network for one grid family (synth.WarmStartFamily)."""

    def __init__(self, family: "synth.WarmStartFamily", channels: int = 64, layers: int = 6, batch: int = 8,
                 sigma: float = 1.0, seed: int = 0, out_scale: float = 0.1, device: str = "cuda:0"):
        torch = _torch()
        self.family = family
        self.batch = batch
        self.dev = torch.device(device)
        self.net = lq2d.WarmStartNet(family.K, family.N, family.T, family.n, channels, layers, batch, sigma)
        self.net.set_params(synth.warmstart_init(self.net.layer_sizes(), seed, out_scale))
        self.problem = None
        self.x0 = None
        self.targets = None
        self.couplings = None
        self.iterations = None

    # -- data ----------------------------------------------------------
    def _problem_for(self, g):
        torch = _torch()
        arrs = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(self.dev) for a in g.arrays()]
        if self.problem is None:
            self.problem = lq2d.Problem.from_device(g.K, g.N, g.T, g.n, g.m, *arrs)
        else:
            self.problem.update_device(*arrs)
        return self.problem

    def generate(self, seeds, tol: float = 1e-6, precision: int = 1, S: int = 2, L: int = 2):
        """Solves each instance (zero start) and keeps x0, c and the costates
        on the device as training pairs.  Returns the wall time."""
        torch = _torch()
        f = self.family
        count = len(seeds)
        self.x0 = torch.empty((count, f.K * f.N, f.n), dtype=torch.float64, device=self.dev)
        self.targets = torch.empty((count, f.T + 1, f.K * f.N, f.n), dtype=torch.float64, device=self.dev)
        self.couplings = np.empty(count)
        self.iterations = np.empty(count, dtype=np.int64)
        t0 = time.perf_counter()
        for idx, seed in enumerate(seeds):
            c, x0 = f.instance_params(seed)
            prob = self._problem_for(f.grid(c, x0))
            prob.set_precision(precision)
            out = prob.solve_device(tol, S, L, 100000, costate=self.targets[idx])
            self.iterations[idx] = out["iterations"]
            self.x0[idx].copy_(torch.from_numpy(x0))
            self.couplings[idx] = c
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def _solve_group(self, chunk, slot: int, tol: float, S: int, L: int):
        """Solves the seeds of `chunk` as one multi-right-hand-side problem
        with the coupling of chunk[0] (each seed keeps its own x0) and writes
        x0, c and the costates to pair slots slot, slot + 1, ...; returns the
        iteration count of each pair."""
        torch = _torch()
        f = self.family
        c, x0_first = f.instance_params(chunk[0])
        for k, sd in enumerate(chunk):
            self.x0[slot + k].copy_(torch.from_numpy(f.instance_params(sd)[1]))
            self.couplings[slot + k] = c
        prob = self._problem_for(f.grid(c, x0_first))
        out = prob.solve_multi_device(len(chunk), self.x0[slot:slot + len(chunk)], tol, S, L, 100000,
                                      costate=self.targets[slot:slot + len(chunk)])
        return out["iterations"]

    def generate_grouped(self, seeds, tol: float = 1e-6, S: int = 2, L: int = 2, group: int = 32):
        """As generate, 32 instances per solve: consecutive seeds form groups
        of `group` that share the coupling drawn by the group's first seed
        (each keeps its own x0), and each group is one multi-right-hand-side
        solve (lq2d_solve_multi_device).  The pairs still cover the family:
        c is uniform over groups, x0 standard normal per pair.  Returns the
        wall time."""
        torch = _torch()
        f = self.family
        seeds = list(seeds)
        count = len(seeds)
        self.x0 = torch.empty((count, f.K * f.N, f.n), dtype=torch.float64, device=self.dev)
        self.targets = torch.empty((count, f.T + 1, f.K * f.N, f.n), dtype=torch.float64, device=self.dev)
        self.couplings = np.empty(count)
        self.iterations = np.empty(count, dtype=np.int64)
        t0 = time.perf_counter()
        for start in range(0, count, group):
            chunk = seeds[start:start + group]
            self.iterations[start:start + len(chunk)] = self._solve_group(chunk, start, tol, S, L)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def fit_online(self, seeds, steps_per_group: int, tol: float = 1e-6, S: int = 2, L: int = 2,
                   group: int = 32, buffer: int = 2048, lr: float = 1e-3, lr_final: float = 1e-4,
                   seed: int = 0):
        """Training without storing every target (20k FP64 solutions of the
        128 x 128 x 100 family take about 1 TB): consecutive seeds are solved
        `group` at a time (the rule of generate_grouped), their pairs go into
        a ring buffer of `buffer` pairs on the device, and after each group
        `steps_per_group` Adam steps sample minibatches from the pairs in the
        buffer.  The learning rate decays geometrically from lr to lr_final
        over all steps.  Returns (losses, generation seconds, training
        seconds, pairs generated)."""
        torch = _torch()
        f = self.family
        seeds = list(seeds)
        if buffer % group != 0:
            raise ValueError("buffer must be a multiple of group")
        cap = min(buffer, len(seeds) + (-len(seeds)) % group)
        self.x0 = torch.empty((cap, f.K * f.N, f.n), dtype=torch.float64, device=self.dev)
        self.targets = torch.empty((cap, f.T + 1, f.K * f.N, f.n), dtype=torch.float64, device=self.dev)
        self.couplings = np.zeros(cap)
        its = []
        groups = (len(seeds) + group - 1) // group
        total = groups * steps_per_group
        rng = np.random.default_rng(seed)
        b = self.batch
        xb = torch.empty((b,) + tuple(self.x0.shape[1:]), dtype=torch.float64, device=self.dev)
        tb = torch.empty((b,) + tuple(self.targets.shape[1:]), dtype=torch.float64, device=self.dev)
        losses = []
        gen_s = train_s = 0.0
        step = 0
        for gi in range(groups):
            chunk = seeds[gi * group:(gi + 1) * group]
            slot = (gi * group) % cap
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its.extend(self._solve_group(chunk, slot, tol, S, L))
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            gen_s += t1 - t0
            avail = min(cap, gi * group + len(chunk))
            for _ in range(steps_per_group):
                idx = rng.choice(avail, size=min(b, avail), replace=False)
                if len(idx) < b:
                    idx = np.resize(idx, b)
                rate = lr * (lr_final / lr) ** (step / max(1, total - 1))
                losses.append(self._train_step(idx, xb, tb, rate))
                step += 1
            torch.cuda.synchronize()
            train_s += time.perf_counter() - t1
        self.iterations = np.array(its, dtype=np.int64)
        return np.array(losses), gen_s, train_s, len(seeds)

    # -- training --------------------------------------------------------
    def _train_step(self, idx, xb, tb, rate: float) -> float:
        """One Adam step on the stored pairs idx (gathered into xb, tb)."""
        torch = _torch()
        ii = torch.from_numpy(idx).to(self.dev)
        torch.index_select(self.x0, 0, ii, out=xb)
        torch.index_select(self.targets, 0, ii, out=tb)
        return self.net.train_step_device(len(idx), xb, self.couplings[idx], tb, rate)

    def fit(self, steps: int, lr: float = 1e-3, lr_final: float = 1e-4, seed: int = 0, log_every: int = 0):
        """Adam steps on random minibatches of the generated pairs, with the
        learning rate decayed geometrically from lr to lr_final.  Returns the
        per-step losses."""
        count = self.x0.shape[0]
        rng = np.random.default_rng(seed)
        losses = []
        b = min(self.batch, count)
        torch = _torch()
        xb = torch.empty((b,) + tuple(self.x0.shape[1:]), dtype=torch.float64, device=self.dev)
        tb = torch.empty((b,) + tuple(self.targets.shape[1:]), dtype=torch.float64, device=self.dev)
        for s in range(steps):
            idx = rng.choice(count, size=b, replace=False)
            rate = lr * (lr_final / lr) ** (s / max(1, steps - 1))
            losses.append(self._train_step(idx, xb, tb, rate))
            if log_every and (s % log_every == 0 or s + 1 == steps):
                print("step %d loss %.4e lr %.2e" % (s, losses[-1], rate), flush=True)
        return np.array(losses)

    # -- use -------------------------------------------------------------
    def guess(self, c: float, x0_dev, out=None):
        """delta^(0) [T+1][K*N][n] of one instance (device tensor)."""
        torch = _torch()
        f = self.family
        if out is None:
            out = torch.empty((f.T + 1, f.K * f.N, f.n), dtype=torch.float64, device=self.dev)
        self.net.forward_device(1, x0_dev, [c], out)
        return out

    def solve(self, seed: int, tol: float = 1e-8, warm: bool = True, precision: int = 0, S: int = 2, L: int = 2):
        """Solves instance `seed` from the network's guess (warm) or from zero;
        returns iterations, relative KKT residual, the costate and the time
        of guess + solve (seconds, wall clock around synchronised calls)."""
        torch = _torch()
        f = self.family
        c, x0 = f.instance_params(seed)
        prob = self._problem_for(f.grid(c, x0))
        prob.set_precision(precision)
        lam = torch.empty((f.T + 1, f.K * f.N, f.n), dtype=torch.float64, device=self.dev)
        x0d = torch.from_numpy(x0).to(self.dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d0 = self.guess(c, x0d) if warm else None
        out = prob.solve_device(tol, S, L, 100000, delta0=d0, costate=lam)
        torch.cuda.synchronize()
        return dict(iterations=out["iterations"], rel_kkt=out["rel_kkt"], costate=lam,
                    seconds=time.perf_counter() - t0, status=out["status"])

    def close(self):
        if self.problem is not None:
            self.problem.close()
        self.net.close()
