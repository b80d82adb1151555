"""Exact i.i.d. draws of Fourier modes from the importance measures of Eq. (59), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Target (Eq. 59): P(k) = calF(k) Fhat(k) / S over k = 2 pi (m_x/L_x, m_y/L_y, m_z/L_z),
m in Z^3 \\ {0}, with Fhat of Eq. (54), calF the Debye-Hueckel correction of Eq. (62)
and S = sum_{k != 0} calF Fhat.

Procedure (the reading of the sampling step of Algorithm 2 used throughout; the
paper's own sampler is Metropolis-Hastings, Sec. 4.3, while the variance lemma
(Lemma 4.1) assumes i.i.d. draws, which this gives exactly):
  Fhat(k) = sum_m A_m prod_a g_{m,a}(n_a),  A_m = pi^{3/2} h w_m f(t_m,0) e^{-3 t_m/2},
  g_{m,a}(n) = exp(-(2 pi n / L_a)^2 / (4 b_m)),  b_m = e^{t_m}.
  1. pick the Gaussian m with probability proportional to A_m prod_a theta_{m,a},
     theta_{m,a} = sum_n g_{m,a}(n)          (alias table over m);
  2. per axis draw n_a with probability g_{m,a}(n_a) / theta_{m,a}
     (alias table over |n_a| <= nmax_{m,a}, where g < 1e-18 beyond);
  3. if n = 0, start the attempt over;
  4. accept with probability calF(k) / sum_j q_j^2 (calF increases with |k| towards
     sum q^2), else start over; the test u < kT V / (kT V + Q2/t), t = k^2 + lambda^-2, is
     evaluated as u (kT V t + Q2) < kT V t.
Accepted modes are distributed as P(k).

DEBYE (Eq. 62 with the Debye wavenumber of Gaussian units, 4 pi sum q^2 / (k_B T V)) is the
same procedure with sum q^2 replaced by 4 pi sum q^2 in the acceptance ratio of step 4:
calF_D(k) = kT V / (kT V / sum q^2 + 4 pi / (k^2 + lambda^-2)) also rises to sum q^2.

The other two corrections compared in Sec. 5 (Fig. 9) use the same machinery:
  calF = 1:    steps 1-3 only (every nonzero draw is accepted);
  calF = k^2:  k^2 Fhat(k) = sum_m A_m sum_a k_a^2 g_{m,a}(n_a) prod_{b != a} g_{m,b}(n_b) is a
               mixture over (m, a) with weights A_m sigma_{m,a} prod_{b != a} theta_{m,b},
               sigma_{m,a} = sum_n (2 pi n / L_a)^2 g_{m,a}(n); step 1 picks (m, a) (index
               3 m + a), axis a is drawn from the k_a^2-weighted table (whose n = 0 entry has
               weight 0, so k != 0) and the other axes from the plain tables; no rejection.

Random numbers: Philox4x32-10, key = (seed lo, seed hi), counter = (slot l, 8*attempt + j,
draw lo, draw hi) with j = 0 for the Gaussian index, j = 1, 2, 3 for the axes, j = 4 for
the acceptance test.  An alias draw from words (x0, x1, x2, x3) takes the index
floor((x0 2^32 + x1) n / 2^64) and keeps it when u53(x2, x3) < prob[index], else takes
alias[index].  Alias tables follow Vose (1991) with both work lists used as stacks,
filled in ascending index order.  The same layout lets a replay reproduce another
implementation's draws from the same seed.
"""
from __future__ import annotations

import math

import numpy as np

from . import philox
from .sog import SOG, f_tr

LN_1E18 = 41.44653167389282      # ln(1e18): 1-D tables stop where g < 1e-18
TWO_PI = 6.283185307179586
MAX_ATTEMPTS = 1 << 20


def vose_alias(weights):
    """Alias table (prob, alias) for the discrete distribution proportional to weights."""
    w = [float(x) for x in weights]
    n = len(w)
    total = 0.0
    for x in w:
        total += x
    scaled = [(x * n) / total for x in w]
    prob = [0.0] * n
    alias = list(range(n))
    small = [i for i in range(n) if scaled[i] < 1.0]
    large = [i for i in range(n) if scaled[i] >= 1.0]
    while small and large:
        lo = small.pop()
        g = large.pop()
        prob[lo] = scaled[lo]
        alias[lo] = g
        scaled[g] = (scaled[g] + scaled[lo]) - 1.0
        if scaled[g] < 1.0:
            small.append(g)
        else:
            large.append(g)
    while large:
        prob[large.pop()] = 1.0
    while small:
        prob[small.pop()] = 1.0
    return np.asarray(prob, dtype=np.float64), np.asarray(alias, dtype=np.int64)


ADAPTIVE, UNIFORM, K2, DEBYE = 0, 1, 2, 3


class ModeSampler:
    """Tables for drawing k from P(k) for one (SOG, box, k_B T, charges) state and one
    measure (ADAPTIVE: calF of Eq. 62; UNIFORM: calF = 1; K2: calF = k^2)."""

    def __init__(self, sog: SOG, L, kT: float, Q2: float, kind: int = ADAPTIVE):
        self.kind = int(kind)
        self.sog = sog
        self.L = [float(x) for x in L]
        self.kT = float(kT)
        self.Q2 = float(Q2)
        self.V = (self.L[0] * self.L[1]) * self.L[2]
        self.tpl = [TWO_PI / x for x in self.L]
        self.inv_lam2 = 1.0 / (sog.lam * sog.lam)
        t = sog.t
        wt = sog.weights
        self.b = [math.exp(float(x)) for x in t]
        self.A = [sog.h * float(wt[i]) * math.pi ** 1.5 * float(f_tr(float(t[i]), 0.0, sog.lam))
                  * math.exp(-1.5 * float(t[i])) for i in range(len(t))]
        self.axis = []       # per mixture component: list of 3 (nmax, prob, alias)
        mix = []
        for i, b in enumerate(self.b):
            plain, sq = [], []
            theta, sigma = [], []
            for a in range(3):
                nmax = int(math.ceil(math.sqrt(4.0 * b * LN_1E18) / self.tpl[a]))
                g, g2 = [], []
                for n in range(-nmax, nmax + 1):
                    kk = self.tpl[a] * n
                    e = math.exp(-(kk * kk) / (4.0 * b))
                    g.append(e)
                    g2.append((kk * kk) * e)
                th = 0.0
                for x in g:
                    th += x
                sg = 0.0
                for x in g2:
                    sg += x
                prob, alias = vose_alias(g)
                plain.append((nmax, prob, alias))
                theta.append(th)
                if self.kind == K2:
                    prob2, alias2 = vose_alias(g2)
                    sq.append((nmax, prob2, alias2))
                    sigma.append(sg)
            if self.kind == K2:
                for a in range(3):
                    tabs = [sq[c] if c == a else plain[c] for c in range(3)]
                    self.axis.append(tabs)
                    w = self.A[i] * sigma[a]
                    for c in range(3):
                        if c != a:
                            w = w * theta[c]
                    mix.append(w)
            else:
                self.axis.append(plain)
                mix.append(self.A[i] * ((theta[0] * theta[1]) * theta[2]))
        self.mix_prob, self.mix_alias = vose_alias(mix)

    def accept_ratio(self, k2):
        """calF(k)/sum q^2 = kT V / (kT V + Q2/(k^2 + lambda^-2)), with 4 pi Q2 for DEBYE."""
        A = self.kT * self.V
        Q2 = (4.0 * math.pi) * self.Q2 if self.kind == DEBYE else self.Q2
        return A / (A + Q2 * (1.0 / (k2 + self.inv_lam2)))

    def accepts(self, u, k2):
        """Step 4, u < calF(k)/sum q^2 = A / (A + Q2/t) with A = kT V, t = k^2 + lambda^-2,
        evaluated without division as u (A t + Q2) < A t (IEEE double operations)."""
        A = self.kT * self.V
        Q2 = (4.0 * math.pi) * self.Q2 if self.kind == DEBYE else self.Q2
        At = A * (k2 + self.inv_lam2)
        return u * (At + Q2) < At

    def k2_of(self, m):
        m = np.asarray(m, dtype=np.float64)
        kx = self.tpl[0] * m[..., 0]
        ky = self.tpl[1] * m[..., 1]
        kz = self.tpl[2] * m[..., 2]
        return (kx * kx + ky * ky) + kz * kz

    def _alias_pick(self, words, prob, alias, n):
        i = philox.index_below(words[0], words[1], n)
        u = philox.u53(words[2], words[3])
        return np.where(u < prob[i], i, alias[i])

    def draw(self, seed: int, draw_index: int, P: int):
        """P i.i.d. modes (int32 [P,3]) and the attempt count each slot used."""
        k0 = np.uint64(seed & 0xFFFFFFFF)
        k1 = np.uint64((seed >> 32) & 0xFFFFFFFF)
        c2 = np.uint64(draw_index & 0xFFFFFFFF)
        c3 = np.uint64((draw_index >> 32) & 0xFFFFFFFF)
        out = np.zeros((P, 3), dtype=np.int64)
        attempts = np.zeros(P, dtype=np.int64)
        todo = np.arange(P, dtype=np.int64)
        att = 0
        while todo.size:
            if att >= MAX_ATTEMPTS:
                raise RuntimeError("sampler exceeded the attempt limit")
            slot = todo.astype(np.uint64)
            words = [philox.philox4x32_10(slot, np.uint64(8 * att + j), c2, c3, k0, k1) for j in range(5)]
            mi = self._alias_pick(words[0], self.mix_prob, self.mix_alias, len(self.mix_prob))
            n = np.zeros((todo.size, 3), dtype=np.int64)
            for a in range(3):
                for g in np.unique(mi):
                    sel = mi == g
                    nmax, prob, alias = self.axis[g][a]
                    wsel = [x[sel] for x in words[1 + a]]
                    n[sel, a] = self._alias_pick(wsel, prob, alias, 2 * nmax + 1) - nmax
            nonzero = np.any(n != 0, axis=1)
            if self.kind in (ADAPTIVE, DEBYE):
                u = philox.u53(words[4][0], words[4][1])
                ok = nonzero & self.accepts(u, self.k2_of(n))
            else:
                ok = nonzero
            out[todo[ok]] = n[ok]
            attempts[todo[ok]] = att + 1
            todo = todo[~ok]
            att += 1
        return out.astype(np.int32), attempts

    # --- exact measure (for pins) ---
    def calF(self, k2):
        k2 = np.asarray(k2, dtype=np.float64)
        if self.kind == UNIFORM:
            return np.ones_like(k2)
        if self.kind == K2:
            return k2
        if self.kind == DEBYE:
            return self.kT * self.V / (self.kT * self.V / self.Q2 + (4.0 * math.pi) / (k2 + self.inv_lam2))
        return self.kT * self.V / (self.kT * self.V / self.Q2 + 1.0 / (k2 + self.inv_lam2))

    def fhat(self, k2):
        k2 = np.asarray(k2, dtype=np.float64)
        return sum(self.A[i] * np.exp(-k2 / (4.0 * self.b[i])) for i in range(len(self.b)))

    def all_modes(self, tail=1e-17):
        """Every m != 0 with Fhat(k) above tail * Fhat(0)-scale cutoff: k^2 <= 4 b_max ln(1/tail)."""
        kmax2 = 4.0 * max(self.b) * math.log(1.0 / tail)
        nm = [int(math.floor(math.sqrt(kmax2) / self.tpl[a])) + 1 for a in range(3)]
        g = [np.arange(-nm[a], nm[a] + 1) for a in range(3)]
        mx, my, mz = np.meshgrid(*g, indexing="ij")
        m = np.stack([mx.ravel(), my.ravel(), mz.ravel()], axis=1)
        m = m[np.any(m != 0, axis=1)]
        m = m[self.k2_of(m) <= kmax2]
        return m.astype(np.int64)


MH_TAG = 0x80000000          # top bit of the fourth counter word: the chains' own stream
MH_T_BITS = 29               # proposal index t enters as (8 (t mod 2^29) + j, t >> 29)


class MHChains:
    """P independent Metropolis-Hastings chains on Z^3 \\ {0} whose stationary measure is
    P(k) of Eq. (59): the sampler Sec. 4.3 names for drawing the batch.

    The paper names the method only.  Reading used here: an independence sampler whose
    proposal Q is the exact draw of steps 1-2 of ModeSampler (the Gaussian mixture of Fhat,
    or of k^2 Fhat for calF = k^2) and whose acceptance probability is
        alpha(k -> k') = min(1, a(k') / a(k)),   a(k) = P(k) / Q(k) (up to a constant),
    so a(k) = calF(k) / sum q^2 for the adaptive measures and a = 1 otherwise (every move
    is accepted and the chain is i.i.d.).  A proposal k' = 0 is rejected (the chain stays).
    With A = kT V, t = k^2 + lambda^-2 and At = A t, the test u < a(k')/a(k) is evaluated
    without division as (u At)(At' + Q2) < At' (At + Q2) in IEEE double operations.

    Chain l's proposal number t (counted from its start, never reset) uses the Philox words
    counter = (l, 8 (t mod 2^29) + j, t >> 29, 2^31), key = seed: j = 0 mixture, j = 1..3
    axes, j = 4 the uniform u.  At its first evaluation a chain takes its first nonzero
    proposal as its state and then makes `burnin` more proposals; every later evaluation
    makes `sweeps` proposals.  The evaluation's batch is the P chain states."""

    def __init__(self, sampler: "ModeSampler", P: int, sweeps: int = 1, burnin: int = 64):
        self.s = sampler
        self.P = int(P)
        self.sweeps = int(sweeps)
        self.burnin = int(burnin)
        self.m = np.zeros((self.P, 3), dtype=np.int64)
        self.t = np.zeros(self.P, dtype=np.int64)
        self.started = False
        self.accepted = 0
        self.proposed = 0

    def _words(self, seed: int, slots, t):
        k0 = np.uint64(seed & 0xFFFFFFFF)
        k1 = np.uint64((seed >> 32) & 0xFFFFFFFF)
        slots = np.asarray(slots, dtype=np.uint64)
        t = np.asarray(t, dtype=np.uint64)
        lo = t & np.uint64((1 << MH_T_BITS) - 1)
        hi = t >> np.uint64(MH_T_BITS)
        return [philox.philox4x32_10(slots, np.uint64(8) * lo + np.uint64(j), hi, np.uint64(MH_TAG), k0, k1)
                for j in range(5)]

    def _propose(self, seed: int, slots):
        """Proposal n ([len(slots), 3]) and u of each chain's next proposal."""
        s = self.s
        words = self._words(seed, slots, self.t[slots])
        mi = s._alias_pick(words[0], s.mix_prob, s.mix_alias, len(s.mix_prob))
        n = np.zeros((len(slots), 3), dtype=np.int64)
        for a in range(3):
            for g in np.unique(mi):
                sel = mi == g
                nmax, prob, alias = s.axis[g][a]
                wsel = [x[sel] for x in words[1 + a]]
                n[sel, a] = s._alias_pick(wsel, prob, alias, 2 * nmax + 1) - nmax
        self.t[slots] += 1
        return n, philox.u53(words[4][0], words[4][1])

    def accepts(self, u, k2_cur, k2_new):
        """u < a(k')/a(k) as (u At)(At' + Q2) < At' (At + Q2)."""
        s = self.s
        if s.kind not in (ADAPTIVE, DEBYE):
            return np.ones(np.shape(u), dtype=bool)
        A = s.kT * s.V
        Q2 = (4.0 * math.pi) * s.Q2 if s.kind == DEBYE else s.Q2
        At = A * (k2_cur + s.inv_lam2)
        Atn = A * (k2_new + s.inv_lam2)
        return (u * At) * (Atn + Q2) < Atn * (At + Q2)

    def _sweep(self, seed: int):
        slots = np.arange(self.P)
        n, u = self._propose(seed, slots)
        ok = np.any(n != 0, axis=1) & self.accepts(u, self.s.k2_of(self.m), self.s.k2_of(n))
        self.m[ok] = n[ok]
        self.accepted += int(np.sum(ok))
        self.proposed += self.P

    def draw(self, seed: int):
        """The P modes (int32 [P, 3]) of the next force evaluation."""
        if not self.started:
            todo = np.arange(self.P)
            tries = 0
            while todo.size:
                if tries >= MAX_ATTEMPTS:
                    raise RuntimeError("MH chain start exceeded the attempt limit")
                n, _ = self._propose(seed, todo)
                nz = np.any(n != 0, axis=1)
                self.m[todo[nz]] = n[nz]
                todo = todo[~nz]
                tries += 1
            self.started = True
            for _ in range(self.burnin):
                self._sweep(seed)
        else:
            for _ in range(self.sweeps):
                self._sweep(seed)
        return self.m.astype(np.int32)
