"""Helpers that run the same seeded case through the GPU library and the
oracle.  Inputs come from paper_0809_4958_gb300.inputs (random draws) and from
the oracle's generator (FP64 boundary samples and initial field); nothing the
oracle sees comes from the GPU."""
from __future__ import annotations

import numpy as np

import oracle
from paper_0809_4958_gb300 import inputs


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def interior(u, periodic=(False, False, False)):
    sl = [slice(None)]
    for a in (2, 1, 0):  # array axes are z, y, x
        sl.append(slice(None) if periodic[a] else slice(1, -1))
    return u[tuple(sl)]


class Case:
    """One box: synthetic Kolmogorov-spectrum boundary, optional chain."""

    def __init__(self, E, tau, nsteps, seed=0, M=64, k_max=None, K=1, time_interp=0, periodic=(False, False, False),
                 accel=(0.0, 0.0, 0.0), nbeads=0, kT=0.0, n_md=50, pin_com=2, chain_seed=7, vel0=None, zoom=1):
        self.E, self.tau, self.nsteps, self.K, self.zoom = E, tau, nsteps, K, zoom
        self.time_interp, self.periodic, self.accel = time_interp, tuple(periodic), tuple(accel)
        self.modes = inputs.mode_table(seed, M, 1.0, float(k_max or E // 2), E)
        self.J = nsteps // K + 4
        self.samples = oracle.face_samples(self.modes, E, K, 0, self.J, zoom)
        self.u0 = oracle.volume_field(self.modes, E, 0.0, zoom)
        self.nbeads, self.kT, self.n_md, self.pin_com, self.chain_seed = nbeads, kT, n_md, pin_com, chain_seed
        self.pos0 = inputs.chain_start(seed + 100, nbeads, E) if nbeads else None
        self.vel0 = vel0

    def oracle_box(self, storage=oracle.STORE_F64):
        return oracle.BoxParams(E=self.E, tau=self.tau, periodic=self.periodic, accel=self.accel,
                                time_interp=self.time_interp, K=self.K, storage=storage, zoom=self.zoom)

    def oracle_chain(self, box_id=0):
        if not self.nbeads:
            return None
        return oracle.ChainParams(nbeads=self.nbeads, kT=self.kT, seed=self.chain_seed, n_md=self.n_md,
                                  pin_com=self.pin_com, box_id=box_id)

    def run_oracle(self, nsteps=None, storage=oracle.STORE_F64):
        sim = oracle.Sim(self.oracle_box(storage), self.u0, self.samples, self.oracle_chain(), self.pos0, self.vel0)
        st = sim.run(self.nsteps if nsteps is None else nsteps)
        assert st == 0, st
        return sim

    # ---- GPU side ----
    def gpu_desc(self, lbt):
        return lbt.box_desc(self.E, self.tau, self.periodic, self.time_interp, self.K, self.nbeads, 1.0, self.accel,
                            zoom=self.zoom)

    def gpu_chain(self, lbt):
        return lbt.chain_desc(self.nbeads, kT=self.kT, seed=self.chain_seed, n_md=self.n_md, pin_com=self.pin_com)


class GpuRunner:
    """Drives boxes of a Tracers context step by step, pushing each box's
    boundary samples (uploaded once to the device) as they are needed."""

    def __init__(self, lbt, torch, cases, storage, ring_slots=None):
        self.lbt, self.torch, self.cases = lbt, torch, cases
        if ring_slots is None:
            self.tr = lbt.Tracers([c.gpu_desc(lbt) for c in cases], storage)
        else:
            self.tr = lbt.Tracers([c.gpu_desc(lbt) for c in cases], storage, ring_slots=ring_slots)
        real = self.tr.real
        self.dev_samples = [torch.from_numpy(c.samples).to("cuda", real) for c in cases]
        u0s = [torch.from_numpy(c.u0).to("cuda", real).contiguous() for c in cases]
        torch.cuda.synchronize()  # uploads ran on the current stream, the context uses its own
        self.pushed = [-1] * len(cases)
        for b, c in enumerate(cases):
            self.tr.lb_init(b, u0s[b])
            if c.nbeads:
                v0 = None if c.vel0 is None else np.ascontiguousarray(c.vel0, np.float64)
                self.tr.chain_couple(b, c.gpu_chain(lbt), np.ascontiguousarray(c.pos0), v0)
        self.tr.lb_sync()
        self.n = 0

    def _need(self, c, n):
        j = n // c.K
        return j + 1 if c.time_interp == 0 else j + 2

    def push_for(self, n):
        for b, c in enumerate(self.cases):
            if all(c.periodic):
                continue
            while self.pushed[b] < self._need(c, n):
                j = self.pushed[b] + 1
                self.tr.lb_set_boundary(b, j, self.dev_samples[b][j])
                self.pushed[b] = j

    def step(self, k=1):
        for _ in range(k):
            self.push_for(self.n)
            self.tr.lb_step(1)
            self.n += 1
