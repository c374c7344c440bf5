"""Test-side stand-ins for the sharded transform's device steps, built from
the oracle (Algorithm 1 / Algorithm 2 on each column and row vector, the
definition by Horner for E_q and the known part of the last row) and the
row/column identity F(omega_{rho R + j}) = sum_q (omega_{rho R} omega_j)^q
C_q(omega_rho) (Section 1.3's split; omega_{rho R} omega_j = omega_{rho R +
j} for disjoint bits).  They let the host logic of
paper_1001_5272_gb300/shard.py run on CPU ranks (gloo) with an
independently computed data plane.  Test infrastructure only."""

import numpy as np

from oracle import field as F
from oracle import native as NV


class CpuOps:
    def __init__(self, pid, layout):
        self.pid, self.L = pid, layout
        self.p = F.PRIME_BY_ID[pid].p

    def _pows(self, w, count):
        out, v = [], 1
        for _ in range(count):
            out.append(v)
            v = v * w % self.p
        return out

    def columns(self, inverse, which, block, part, E):
        L, pid = self.L, self.pid
        B = block.numpy().view(np.uint64)
        Ev = E.numpy().view(np.uint64) if E is not None else None
        lc = L.long_cols(part)
        wa = NV.omega(pid, L.a)
        for j in range(L.W):
            long = j < lc
            m = L.a + 1 if long else L.a
            if not inverse:
                col = B[:m, j].copy()
                if not long and Ev is not None and L.b > 0:
                    Ev[j] = NV.eval_at(pid, col, wa) if m else 0
                if m:
                    B[:m, j] = NV.alg1_tft(pid, col)
            elif which == 0 and not long:
                col = NV.alg2_itft(pid, B[:m, j]) if m else B[:0, j]
                if m:
                    B[:m, j] = col
                if Ev is not None and L.b > 0:
                    Ev[j] = NV.eval_at(pid, col, wa) if m else 0
            elif which == 1 and long:
                B[:m, j] = NV.alg2_itft(pid, B[:m, j])

    def rows(self, inverse, rows, rho_begin):
        L, pid, p = self.L, self.pid, self.p
        Rw = rows.numpy().view(np.uint64)
        for i in range(Rw.shape[0]):
            w = NV.omega(pid, (rho_begin + i) * L.R)
            if not inverse:
                pw = self._pows(w, L.R)
                d = np.array([int(v) * q % p for v, q in zip(Rw[i], pw)],
                             dtype=np.uint64)
                Rw[i] = NV.alg1_tft(pid, d)
            else:
                pw = self._pows(pow(w, p - 2, p), L.R)
                d = NV.alg2_itft(pid, Rw[i])
                Rw[i] = np.array([int(v) * q % p for v, q in zip(d, pw)],
                                 dtype=np.uint64)

    def last_row(self, inverse, row, E):
        L, pid, p = self.L, self.pid, self.p
        b = L.b
        rv = row.numpy().view(np.uint64)
        Ev = E.numpy().view(np.uint64)
        w = NV.omega(pid, L.a * L.R)
        pw = self._pows(w, L.R)
        if not inverse:
            d = np.array([int(rv[q] if q < b else Ev[q]) * pw[q] % p
                          for q in range(L.R)], dtype=np.uint64)
            rv[:b] = NV.alg1_tft(pid, d)[:b]
            return
        # Y_j = D_b(omega_j) + sum_{q >= b} d_q omega_j^q for j < b: take
        # the known part away, then the length-b inverse gives d_q, q < b
        hi = np.array([0] * b + [int(Ev[q]) * pw[q] % p
                                 for q in range(b, L.R)], dtype=np.uint64)
        known = NV.eval_tft_points(pid, hi, np.arange(b, dtype=np.uint64))
        Yp = np.array([(int(rv[j]) - int(known[j])) % p for j in range(b)],
                      dtype=np.uint64)
        d = NV.alg2_itft(pid, Yp)
        inv = self._pows(pow(w, p - 2, p), b)
        rv[:b] = np.array([int(d[q]) * inv[q] % p for q in range(b)],
                          dtype=np.uint64)
