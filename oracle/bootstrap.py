"""Full-slot CKKS bootstrapping on the CPU oracle.  TEST INFRASTRUCTURE ONLY.

ReBoot refreshes weights and velocities with CKKS bootstrapping (Sec. 3,
last paragraph; Alg. 1, the two Bootstrap lines; Sec. 4.3.4) and defers its
construction to Cheon et al. 2018, Bossuat et al. 2021 and Bae et al. 2022.
The paper fixes the structure (ModRaise, homomorphic encoding, a scaled sine
for the modular reduction, homomorphic decoding) and the level budget
tau_bs = 16 (Sec. 5.1, Table 3).  This module writes that textbook procedure out
step by step over the oracle's primitives; every choice the paper leaves open
is named B1..B8 and listed in the design notes:

  B1 ModRaise: centred lift of c0, c1 mod q0 into every limb of Q_L; the
     raised ciphertext is read at scale q0, so its slots are tau(m + q0 I)/q0.
  B2 Slot transform: z = U w with w = p_lo + i p_hi and U[j][k] = zeta^(g_j k)
     (g_j = 5^j mod 2N), because zeta_j^(N/2) = i.  U = S_n ... S_4 S_2 P
     (radix-2 decimation in time on bit-reversed input; stage S_len pairs
     (r, r + len/2) with twiddle exp(2 pi i (5^j mod 4 len) / (4 len))).
     CoeffToSlot applies P U^-1 and SlotToCoeff applies U P^-1, so the
     bit-reversal P is never evaluated (EvalMod is slot-wise).
  B3 The log2(N/2) stages are merged into three levels (group widths as equal
     as possible, the widest at the bottom); a merged level is a matrix with
     diagonals at offsets k * step, evaluated by baby-step giant-step:
     sum_b Rot(sum_a pt_{b,a} * Rot(x, a step), g b step) with
     pt_{b,a} = Rot(diag_{g b + a}, -g b step); baby rotations hoisted.
     Diagonal plaintexts are encoded at the scale of the prime the level drops.
  B4 Factors folded into the constants: 1/(2K) into the first CoeffToSlot level
     (K = 16: slots become t/(2K), t = p/q0); 1/(2 pi) into the first
     SlotToCoeff level.
  B5 Real and imaginary parts: u_re = u + conj(u), u_im = -i (u - conj(u));
     multiplication by +-i is the exact monomial +-X^(N/2); recombination
     v = v_re + i v_im.
  B6 EvalMod: f(u) = cos(2 pi (K u - 1/4) / 2^r), r = 3, by its degree-60
     Chebyshev interpolant on [-1, 1] (Chebyshev nodes, FP64), then r double
     angles c <- 2 c^2 - 1, giving sin(2 pi t).
  B7 Chebyshev evaluation: T_2..T_8 by T_2k = 2 T_k^2 - 1 and
     T_(a+b) = 2 T_a T_b - T_(a-b) in the fixed order below, giants T_16, T_32;
     p = q T_g + r split recursively at the largest g in {32, 16, 8} <= deg p;
     a part of degree < 8 is a leaf sum_k round(c_k q_l S/S_k) T_k dropped to
     one level l, rescaled once, plus round(c_0 S).  Products take the lower
     level of their operands; a sum takes the scale of its first operand.
  B8 Output scale = (scale after SlotToCoeff) * Delta_in / q0.
  B9 Every ciphertext product (B6, B7) is the relinearised product with
     ModDown and rescale merged into one conversion (reading C21).
  B10 In a merged level the giant steps meet before any ModDown: the sum
     inner_0 + sum_b (P sigma_b(inner_b.c0) + KS_acc(sigma_b(inner_b.c1)))
     over Q_l P (KS_acc: ModUp and key inner product, no ModDown) is divided
     by P q_l once (C21), replacing a ModDown per giant rotation and the
     level's rescale.
  B11 Double hoisting: the baby rotations stay over Q_l P as well (x_a =
     (P sigma_a(c0) + acc0, acc1), no ModDown), the giant terms inner_b are
     sums over Q_l P (diagonal plaintexts carry residues mod P), inner_0
     joins the B10 sum as it is and each other inner_b is ModDown'd once
     before its giant rotation.  With the baby steps this cheap, the split
     is g = 2^(w-1) baby steps (16 x 4 at w = 5) instead of 2^ceil(w/2).
  B12 Iterative bootstrapping (Bae et al. 2022, which Sec. 5.1 cites for the
     depth tau_bs): ct1 = Bootstrap(ct) decrypts to m + e1; the difference
     d = align(ct1, level 0, Delta) - ct carries e1, is multiplied by the
     integer 2^k (no level) and bootstrapped again with the same scale label,
     giving ct2 ~ 2^k e1 + e2.  The result 2^k ct1 - ct2, read at scale
     2^k * (ct1's scale), decrypts to m - e2 / 2^k at ct1's level: the
     division by 2^k is a change of the scale label, so no level is spent.
  B13 Sparse slots (n = 2^s < N/2): a message of n slots is the full-slot
     vector of period n, i.e. a polynomial in X^(N/2n).  After ModRaise the
     sub-sum x <- x + Rot(x, n 2^i), i < log2(N/2n), is the trace onto that
     subring: it keeps d = N/(2n) times the subring part (q0 I included) and
     cancels the rest; 1/d joins the first CoeffToSlot level's 1/(2K).  The
     linear levels are the n-slot transforms with their diagonals repeated
     across the N/2 slots; EvalMod and SlotToCoeff are unchanged.
Parity unpinned: nothing here (see tests/test_oracle_bootstrap.py).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import OCt, Oracle

K_RANGE = 16
CHEB_DEGREE = 60
DOUBLE_ANGLES = 3
LEVELS_CTS = 3
LEVELS_STC = 3
EVALMOD_DEPTH = 7 + DOUBLE_ANGLES


# ----------------------------------------------------------------- B2 / B3
def slot_exponents(n_slots: int) -> np.ndarray:
    m = 4 * n_slots
    g = np.ones(n_slots, dtype=np.int64)
    for j in range(1, n_slots):
        g[j] = (g[j - 1] * 5) % m
    return g


def special_dft_matrix(n_slots: int) -> np.ndarray:
    """U[j][k] = zeta^(g_j k), zeta = exp(2 pi i / 4n) (dense; small n only)."""
    m = 4 * n_slots
    g = slot_exponents(n_slots)
    k = np.arange(n_slots)
    return np.exp(2j * np.pi * ((g[:, None] * k[None, :]) % m) / m)


def stage_twiddles(n_slots: int, lenh: int) -> np.ndarray:
    lenq = 8 * lenh
    g = slot_exponents(n_slots)[:lenh]
    return np.exp(2j * np.pi * (g % lenq) / lenq)


def stage_diags(n_slots: int, lenh: int, inverse: bool) -> dict:
    """Diagonals {offset: vector} of butterfly stage S_(2 lenh) or its inverse.
    Forward, per pair (u, v) = (r, r + lenh): u' = u + xi v, v' = u - xi v."""
    n = n_slots
    xi = stage_twiddles(n, lenh)
    r = np.arange(n)
    pos = r % (2 * lenh)
    upper = pos < lenh
    j = np.where(upper, pos, pos - lenh)
    x = xi[j]
    d0 = np.zeros(n, dtype=np.complex128)
    dp = np.zeros(n, dtype=np.complex128)
    dm = np.zeros(n, dtype=np.complex128)
    if not inverse:
        d0[upper] = 1.0
        dp[upper] = x[upper]
        dm[~upper] = 1.0
        d0[~upper] = -x[~upper]
    else:  # u = (u' + v')/2, v = (u' - v')/(2 xi)
        d0[upper] = 0.5
        dp[upper] = 0.5
        dm[~upper] = 0.5 / x[~upper]
        d0[~upper] = -0.5 / x[~upper]
    out = {0: d0}
    for d, v in ((lenh % n, dp), ((-lenh) % n, dm)):  # +lenh and -lenh coincide when lenh = n/2
        out[d] = out[d] + v if d in out else v
    return out


def diag_matmul(a: dict, b: dict, n: int) -> dict:
    """(A B) in diagonal form: C_(d1+d2)[r] += A_d1[r] B_d2[r + d1]."""
    c: dict = {}
    for d1, v1 in a.items():
        for d2, v2 in b.items():
            d = (d1 + d2) % n
            term = v1 * np.roll(v2, -d1)
            c[d] = c[d] + term if d in c else term
    return c


def diag_apply(diags: dict, x: np.ndarray) -> np.ndarray:
    return sum(v * np.roll(x, -d) for d, v in diags.items())


def groups(log_slots: int, levels: int = 3):
    """Stage ranges [s0, s1) of the merged levels, bottom (small strides) first."""
    base, extra = divmod(log_slots, levels)
    widths = [base + (1 if i < extra else 0) for i in range(levels)]
    out, s = [], 0
    for w in widths:
        out.append((s, s + w))
        s += w
    return out


def group_matrix(n_slots: int, s0: int, s1: int, inverse: bool) -> dict:
    """Forward: S_(2^s1) ... S_(2^(s0+1)); inverse: the product of the inverses
    in reverse order."""
    mats = None
    lenhs = [1 << s for s in range(s1 - 1, s0 - 1, -1)]  # leftmost factor first
    if inverse:
        lenhs = lenhs[::-1]
    for lh in lenhs:
        st = stage_diags(n_slots, lh, inverse)
        mats = st if mats is None else diag_matmul(mats, st, n_slots)
    return {d: v for d, v in mats.items() if np.any(np.abs(v) > 0)}


@dataclass
class LinLevel:
    """One merged level evaluated by BSGS at ciphertext level `level`."""
    step: int
    g: int
    diags: dict                      # offset (in slots) -> vector
    level: int = 0
    plan: list = field(default_factory=list)  # [(b, [(a, vector)])] ascending b, a

    def build_plan(self, n_slots: int):
        ks = sorted({(d // self.step) if d // self.step <= (n_slots // self.step) // 2 else
                     d // self.step - n_slots // self.step for d in self.diags})
        by_b: dict = {}
        for k in ks:
            b, a = divmod(k, self.g)
            by_b.setdefault(b, []).append((a, k))
        self.plan = []
        for b in sorted(by_b):
            items = []
            for a, k in sorted(by_b[b]):
                vec = self.diags[(k * self.step) % n_slots]
                items.append((a, np.roll(vec, self.g * b * self.step)))  # Rot(diag, -g b step)
            self.plan.append((b, items))

    def rotations(self, n_slots: int) -> set:
        rs = {a * self.step for _, items in self.plan for a, _ in items if a}
        rs |= {self.g * b * self.step for b, _ in self.plan if b}
        return {r % n_slots for r in rs}


def linear_levels(n_slots: int, inverse: bool):
    log_slots = int(math.log2(n_slots))
    gs = groups(log_slots)
    levels = []
    order = gs[::-1] if inverse else gs  # CtS applies the top group first
    for (s0, s1) in order:
        d = group_matrix(n_slots, s0, s1, inverse)
        w = s1 - s0
        levels.append(LinLevel(step=1 << s0, g=1 << max(w - 1, 0), diags=d))  # B11: 16 x 4 at w = 5
    return levels


# ----------------------------------------------------------------- B6
def chebyshev_coeffs(f, degree: int) -> np.ndarray:
    """Interpolant at the degree+1 Chebyshev nodes: f ~ sum_k c_k T_k on [-1, 1]."""
    nn = degree + 1
    j = np.arange(nn)
    theta = np.pi * (j + 0.5) / nn
    fx = f(np.cos(theta))
    c = np.array([2.0 / nn * np.sum(fx * np.cos(k * theta)) for k in range(nn)])
    c[0] /= 2
    return c


def evalmod_function(k_range: int = K_RANGE, r: int = DOUBLE_ANGLES):
    return lambda u: np.cos(2 * np.pi * (k_range * u - 0.25) / (1 << r))


def chebyshev_eval_plain(c: np.ndarray, x: np.ndarray) -> np.ndarray:
    return np.polynomial.chebyshev.chebval(x, c)


# ----------------------------------------------------------------- plan
@dataclass
class BootPlan:
    n: int
    n_slots: int
    top: int                       # top level index L
    cts: list
    stc: list
    cheb: np.ndarray
    k_range: int = K_RANGE

    @property
    def subsum_steps(self) -> list:
        """B13: rotations by n_slots 2^i, i < log2(N / (2 n_slots)) (none at full slots)."""
        return [self.n_slots << i for i in range(int(math.log2(self.n // (2 * self.n_slots))))]

    def rotation_steps(self) -> list:
        rs = set(self.subsum_steps)
        for lv in self.cts + self.stc:
            rs |= lv.rotations(self.n_slots)
        return sorted(rs)


def make_plan(log_n: int, n_q: int, log_slots: int | None = None) -> BootPlan:
    n = 1 << log_n
    ns = n // 2 if log_slots is None else 1 << log_slots
    top = n_q - 1
    cts = linear_levels(ns, inverse=True)
    stc = linear_levels(ns, inverse=False)
    # B4: fold 1/(2K) into the first CoeffToSlot level and 1/(2 pi) into the first SlotToCoeff level;
    # B13: with sparse slots also 1/d, d = N / (2 n_slots), which the sub-sum multiplies in
    sparse = n // (2 * ns)
    cts[0].diags = {d: v / (2 * K_RANGE * sparse) for d, v in cts[0].diags.items()}
    stc[0].diags = {d: v / (2 * np.pi) for d, v in stc[0].diags.items()}
    for i, lv in enumerate(cts):
        lv.level = top - i
        lv.build_plan(ns)
    for i, lv in enumerate(stc):
        lv.level = top - LEVELS_CTS - EVALMOD_DEPTH - i
        lv.build_plan(ns)
    cheb = chebyshev_coeffs(evalmod_function(), CHEB_DEGREE)
    return BootPlan(n, ns, top, cts, stc, cheb)


def encode_constants(orc: Oracle, plan: BootPlan) -> list:
    """Integer plaintext coefficients of every diagonal, in plan order:
    CoeffToSlot levels, then SlotToCoeff levels; per level ascending giant b,
    then ascending baby a; each encoded at the scale of the level's prime."""
    out = []
    reps = plan.n // (2 * plan.n_slots)  # B13: a sparse diagonal repeats across the N/2 slots
    for lv in plan.cts + plan.stc:
        scale = float(orc.q[lv.level])
        for _, items in lv.plan:
            for _, vec in items:
                out.append(orc.encode(np.tile(vec, reps), scale))
    return out


# ----------------------------------------------------------------- evaluation
class Evaluator:
    """The bootstrapping circuit over the oracle's primitives (B1-B8)."""

    def __init__(self, orc: Oracle, plan: BootPlan, constants: list, cheb=None, levels=None):
        """levels: plan-level indices whose plaintexts are prepared (default:
        all; a single linear level can then run without the others')."""
        self.o = orc
        self.plan = plan
        self.cheb = plan.cheb if cheb is None else np.asarray(cheb, dtype=np.float64)
        self.pts = []  # NTT-domain plaintexts per level
        idx = 0
        for li, lv in enumerate(plan.cts + plan.stc):
            per = []
            for _, items in lv.plan:
                row = []
                for _ in items:
                    if levels is None or li in levels:
                        row.append(orc.pt_ext_from_int(constants[idx], lv.level))  # over Q_l and P (B11)
                    idx += 1
                per.append(row)
            self.pts.append(per)
        n = orc.n
        mono = np.zeros(n, dtype=np.int64)
        mono[n // 2] = 1
        self.mono_i = {}
        self.mono_mi = {}
        self._mono = mono

    # ---- helpers
    def drop(self, ct: OCt, level: int) -> OCt:
        if ct.level == level:
            return ct
        assert level < ct.level
        return OCt(np.ascontiguousarray(ct.data[:, : level + 1]), level, ct.scale)

    def align(self, ct: OCt, level: int, scale: float) -> OCt:
        """Bring ct to `level` at exactly `scale`: when it sits higher, multiply
        by round(scale q_l / ct.scale) at its own level l and rescale (one of
        its spare levels), then drop the rest; at the same level it is kept."""
        if ct.level > level:
            ql = float(self.o.q[ct.level])
            k = round_half_away(scale * ql / ct.scale)
            r = self.o.mul_int(ct, k)
            r.scale = scale * ql
            ct = self.o.rescale(r)
        return self.drop(ct, level)

    def _pair(self, a: OCt, b: OCt):
        if a.level > b.level:
            return self.align(a, b.level, b.scale), b, b.scale
        if b.level > a.level:
            return a, self.align(b, a.level, a.scale), a.scale
        return a, b, a.scale

    def add(self, a: OCt, b: OCt) -> OCt:
        x, y, s = self._pair(a, b)
        r = self.o.add(x, y)
        r.scale = s
        return r

    def sub(self, a: OCt, b: OCt) -> OCt:
        x, y, s = self._pair(a, b)
        r = self.o.sub(x, y)
        r.scale = s
        return r

    def add_const(self, a: OCt, c: float) -> OCt:
        m = np.zeros(self.o.n, dtype=np.int64)
        m[0] = int(round_half_away(c * a.scale))
        return self.o.add_plain(a, self.o.pt_from_int(m, a.level))

    def mul(self, a: OCt, b: OCt) -> OCt:
        """Relinearised product at the lower level, ModDown and rescale merged (C21)."""
        lv = min(a.level, b.level)
        return self.o.mul_relin_rescale(self.drop(a, lv), self.drop(b, lv))

    def times_i(self, a: OCt, sign: int) -> OCt:
        m = self._mono * sign
        r = self.o.mul_plain(a, self.o.pt_from_int(m, a.level), 1.0)
        r.scale = a.scale
        return r

    # ---- B1
    def mod_raise(self, ct: OCt) -> OCt:
        o = self.o
        n, top = o.n, self.plan.top
        q0 = o.q[0]
        c = o.intt(np.ascontiguousarray(ct.data[:, :1]).reshape(2, n), [0, 0])
        cen = c.astype(np.int64)
        cen = np.where(c > (q0 - 1) // 2, (c.astype(object) - q0).astype(np.int64), cen)
        out = np.zeros((2, top + 1, n), dtype=np.uint64)
        for p in range(2):
            res = np.stack([np.mod(cen[p], np.int64(qi)).astype(np.uint64) for qi in o.q[: top + 1]])
            out[p] = o.ntt(res, list(range(top + 1)))
        return OCt(out, top, float(q0))

    def sigma(self, ct: OCt, g: int) -> OCt:
        """sigma_g on both polynomials of an NTT-domain ciphertext (no key switch)."""
        o = self.o
        mods = list(range(ct.level + 1))
        out = np.empty_like(ct.data)
        for p in range(2):
            out[p] = o.ntt(o.automorph_coeff(o.intt(ct.data[p], mods), mods, g), mods)
        return OCt(out, ct.level, ct.scale)

    # ---- B3, B10, B11
    def linear(self, x: OCt, lv: LinLevel, pts) -> OCt:
        """One merged level, double hoisted (readings B10, B11): the baby
        rotations stay over Q_l P (no ModDown): x_0 = P x, x_a = (P sigma_a(c0) +
        acc0, acc1); each giant term inner_b = sum_a pt_{b,a} x_a over Q_l P
        (plaintexts with residues mod P too); inner_0 joins the final sum as it
        is, every other one is ModDown'd (C9), rotated by sigma_b as in B10
        (P sigma_b(c0) + KS_acc(sigma_b(c1))); one merged ModDown-rescale (C21)
        divides the sum by P q_l."""
        o = self.o
        assert x.level >= lv.level, (x.level, lv.level)
        x = self.drop(x, lv.level)
        l = lv.level
        mods = list(range(l + 1))
        emods = o.ext_mods(l)
        ext = len(emods)
        P = math.prod(int(o.moduli[o.n_q + k]) for k in range(o.n_p))
        pmod = [P % int(o.q[t]) for t in mods]
        qcol = np.array([int(q) for q in o.q[: l + 1]], dtype=np.uint64)[:, None]
        extq = np.array([int(o.moduli[m]) for m in emods], dtype=np.uint64)[:, None]
        babies = sorted({a for _, items in lv.plan for a, _ in items})
        rot = [a for a in babies if a]
        x0 = np.zeros((2, ext, o.n), dtype=np.uint64)
        for p in range(2):
            x0[p, : l + 1] = o.mul_scalars(x.data[p], mods, pmod)
        xa = {0: x0}
        if rot:
            xa.update(zip(rot, o.rotate_hoisted_ext(x, [a * lv.step for a in rot])))
        X = np.zeros((2, ext, o.n), dtype=np.uint64)  # the sum over q_0..q_l, P
        base = np.zeros((2, l + 1, o.n), dtype=np.uint64)  # its part P * base on q_0..q_l
        for (b, items), row in zip(lv.plan, pts):
            inner = np.zeros((2, ext, o.n), dtype=np.uint64)
            for (a, _), pt in zip(items, row):
                for p in range(2):
                    inner[p] = (inner[p] + o.mul_elem(xa[a][p], pt, emods)) % extq
            if b == 0:
                X = (X + inner) % extq
                continue
            c = OCt(np.stack([o.moddown(inner[p], l) for p in range(2)]), l, x.scale)
            g = o.galois_elt((lv.g * b * lv.step) % self.plan.n_slots)  # B13: amounts taken mod the slot count
            t = self.sigma(c, g)
            X = (X + o.keyswitch_ext(t.data[1], l, g)) % extq
            base[0] = (base[0] + t.data[0]) % qcol
        for p in range(2):
            X[p, : l + 1] = (X[p, : l + 1] + o.mul_scalars(base[p], mods, pmod)) % qcol
        out = np.stack([o.moddown_rescale(X[p], l) for p in range(2)])
        return OCt(out, l - 1, x.scale * float(o.q[l]) / float(o.q[l]))

    # ---- B7
    def chebyshev_basis(self, t1: OCt) -> dict:
        T = {1: t1}

        def double(k):
            r = self.o.mul_int(self.mul(T[k], T[k]), 2)
            return self.add_const(r, -1.0)

        def combine(a, b):
            r = self.o.mul_int(self.mul(T[a], T[b]), 2)
            return self.sub(r, T[abs(a - b)])

        T[2] = double(1)
        T[3] = combine(1, 2)
        T[4] = double(2)
        T[5] = combine(2, 3)
        T[6] = double(3)
        T[7] = combine(3, 4)
        T[8] = double(4)
        T[16] = double(8)
        T[32] = double(16)
        return T

    def leaf(self, c: np.ndarray, T: dict, target_scale: float) -> OCt:
        o = self.o
        deg = len(c) - 1
        if deg == 0:  # a constant: carried by T_1 with coefficient 0
            c = np.array([c[0], 0.0])
            deg = 1
        ks = [k for k in range(1, deg + 1)]
        lvl = min(T[k].level for k in ks)
        ql = float(o.q[lvl])
        acc = None
        for k in ks:
            tk = self.drop(T[k], lvl)
            kint = int(round_half_away(c[k] * (ql * target_scale / tk.scale)))
            term = o.mul_int(tk, kint)
            acc = term if acc is None else o.add(acc, term)
        acc.scale = ql * target_scale
        acc = o.rescale(acc)
        return self.add_const(acc, float(c[0]))

    @staticmethod
    def split_point(deg: int) -> int:
        return max(gg for gg in (8, 16, 32) if gg <= deg)

    def poly_level(self, deg: int, T: dict) -> int:
        """Level at which poly() returns a polynomial of this degree."""
        if deg < 8:
            return min(T[k].level for k in range(1, max(deg, 1) + 1)) - 1
        g = self.split_point(deg)
        m = min(self.poly_level(deg - g, T), T[g].level)
        return min(m - 1, self.poly_level(g - 1, T))

    def poly(self, c: np.ndarray, T: dict, target_scale: float) -> OCt:
        """sum_k c_k T_k at exactly target_scale (B7)."""
        deg = len(c) - 1
        if deg < 8:
            return self.leaf(c, T, target_scale)
        g = self.split_point(deg)
        q = np.zeros(deg - g + 1)
        r = np.array(c[:g], dtype=np.float64).copy()
        q[0] = c[g]
        for k in range(g + 1, deg + 1):
            q[k - g] = 2 * c[k]
            r[2 * g - k] -= c[k]
        # the quotient targets the scale that makes (quotient * T_g) land on target_scale
        m = min(self.poly_level(deg - g, T), T[g].level)
        q_scale = target_scale * float(self.o.q[m]) / T[g].scale
        prod = self.mul(self.poly(q, T, q_scale), T[g])
        prod.scale = target_scale
        return self.add(prod, self.poly(r, T, target_scale))

    def evalmod(self, u: OCt) -> OCt:
        T = self.chebyshev_basis(u)
        v = self.poly(self.cheb, T, u.scale)
        for _ in range(DOUBLE_ANGLES):
            v = self.add_const(self.o.mul_int(self.mul(v, v), 2), -1.0)
        return v

    # ---- the whole circuit
    def bootstrap(self, ct: OCt) -> OCt:
        o = self.o
        delta = ct.scale
        x = self.mod_raise(self.drop(ct, 0))
        for k in self.plan.subsum_steps:  # B13: the trace onto the subring of the sparse slots
            x = o.add(x, o.rotate(x, k))
        ncts = len(self.plan.cts)
        for i, lv in enumerate(self.plan.cts):
            x = self.linear(x, lv, self.pts[i])
        xc = o.conjugate(x)
        u_re = o.add(x, xc)
        u_im = self.times_i(o.sub(x, xc), -1)
        v_re = self.evalmod(u_re)
        v_im = self.evalmod(u_im)
        v = self.add(v_re, self.times_i(v_im, 1))
        for i, lv in enumerate(self.plan.stc):
            v = self.linear(v, lv, self.pts[ncts + i])
        v.scale = v.scale * delta / float(o.q[0])
        return v


    # ---- B12
    def bootstrap_iterative(self, ct: OCt, log2_k: int) -> OCt:
        """Two bootstraps: the second refreshes 2^k times the first's error."""
        o = self.o
        delta = ct.scale
        ct1 = self.bootstrap(ct)
        d = o.sub(self.align(ct1, 0, delta), self.drop(ct, 0))
        d.scale = delta
        d2 = o.mul_int(d, 1 << log2_k)
        d2.scale = delta
        ct2 = self.bootstrap(d2)
        up = o.mul_int(ct1, 1 << log2_k)
        out = o.sub(up, ct2)
        out.scale = ct1.scale * float(1 << log2_k)
        return out


def round_half_away(x: float) -> int:
    """Nearest integer, ties away from zero (the rule of C's llround)."""
    t = math.trunc(x)
    frac = abs(x - t)  # exact in binary floating point
    if frac >= 0.5:
        t += 1 if x > 0 else -1
    return int(t)


def boot_key_steps(plan: BootPlan) -> list:
    return plan.rotation_steps()
