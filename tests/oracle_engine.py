"""A slice-by-slice engine for the sharded data flow on CPU (test helper).

It runs the unimodal MC-moments Parareal iteration (Def. 3.1) from the
oracle's step functions (fine propagator, restriction, matching, coarse
propagator), one slice at a time, exposing the same phases as the library's
engine (paper_2310_11365_gb300.shard.LibraryEngine): lift, fine phase over a
block of slices, restriction records, driver over all slices, fine outputs.
Run alone it reproduces orc_parareal bit for bit (checked by the tests), so
the sharded runs it takes part in can be compared with the oracle exactly.
"""
import numpy as np

STAT = 32


class OracleEngine:
    def __init__(self, orc, p):
        self.orc, self.p = orc, p
        self.N, self.P = p.N, p.P
        self.K = min(p.max_iter if p.max_iter > 0 else p.N, p.N)

    def comm_device(self):
        import torch
        return torch.device("cpu")

    # -- phases ------------------------------------------------------------
    def lift(self):
        orc, p, N = self.orc, self.p, self.N
        self.u0 = orc.initial(p)
        st0 = orc.restrict(p, self.u0)
        self.count0 = st0["count"][0]
        rho = [(st0["mean"][0], st0["var"][0])]
        for n in range(N):
            _, m, v = orc.coarse(p, [1.0], [rho[n][0]], [rho[n][1]])
            rho.append((m[0], v[0]))
        self.rho = rho
        self.cache = list(rho[1:])
        # the inputs of sweep 1: the lifting T(rho^0_n, u0)
        self.rule = [None] + [("lift", rho[n]) for n in range(1, N + 1)]
        self.out = [None] * N          # F_n of the latest sweep
        self.rec = np.zeros((N, STAT))
        self.hist = [[self._mv(r) for r in rho]]
        self.k = 0

    def _mv(self, r):
        return (r[0], r[1])

    def _input(self, n):
        p = self.p
        if n == 0:
            return self.u0
        kind, (mu, sg) = self.rule[n][0], self.rule[n][1]
        if kind == "lift":
            doit = self.count0 > 0 and sg >= 0.0
            return self.orc.match(p, n, [mu], [sg], [int(doit)], self.u0)
        doit = self.rule[n][2]
        return self.orc.match(p, n, [mu], [sg], [int(doit)], self.out[n - 1])

    def fine(self, lo, hi):
        self.k += 1
        first = max(self.k - 1, lo)
        ins = {n: self._input(n) for n in range(first, hi)}  # from the previous sweep's outputs
        for n in range(first, hi):
            self.out[n] = self.orc.fine(self.p, n, ins[n])
            st = self.orc.restrict(self.p, self.out[n])
            row = np.zeros(STAT)
            row[0], row[1], row[2] = st["count"][0], st["mean"][0], st["var"][0]
            row[10], row[11] = st["gmean"], st["gvar"]
            self.rec[n] = row

    def records(self, lo, hi):
        return self.rec[lo:hi].copy()

    def set_records(self, lo, hi, rows):
        self.rec[lo:hi] = rows

    def coarse(self):
        """The driver of sweep k over all slices (the oracle's order of
        operations), then the convergence test."""
        orc, p, N = self.orc, self.p, self.N
        new = [self.rho[0]]
        rule = [None]
        for n in range(N):
            _, am_, av_ = orc.coarse(p, [1.0], [new[n][0]], [new[n][1]])
            a = (am_[0], av_[0])
            bm, bv = self.rec[n][1], self.rec[n][2]
            am = bm + (a[0] - self.cache[n][0])
            av = bv + (a[1] - self.cache[n][1])
            if av >= 0.0:
                new.append((am, av))
                rule.append(("match", (am, av), 1))
            else:
                new.append((bm, bv))
                rule.append(("match", (bm, bv), 0))
            self.cache[n] = a
        change = max(max(abs(x[0] - y[0]), abs(x[1] - y[1])) for x, y in zip(new, self.rho))
        self.rho, self.rule = new, rule
        self.hist.append([self._mv(r) for r in new])
        return change < self.p.tol or self.k >= self.K

    def empty_output(self):
        import torch
        return torch.empty(self.P, dtype=torch.float64)

    def output(self, n):
        import torch
        return torch.from_numpy(self.out[n].copy())

    def set_output(self, n, ensemble):
        self.out[n] = ensemble.cpu().numpy().astype(np.float64).copy()

    def moments(self):
        return np.array(self.hist)
