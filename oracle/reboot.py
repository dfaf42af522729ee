"""ReBoot RE-Block training step on the CPU oracle.  TEST INFRASTRUCTURE ONLY.

Follows the paper step by step:
  * packing (Sec. 4.1): expanded / repeated vectors, row-wise / column-wise
    matrices, zero-padded to r x c with r c = N/2, flattened row-major;
  * sum across rows (Eq. sumrows): log2 r steps s <- s + Rot(s, c 2^(log2 r - 1 - t));
  * sum across columns (Eq. sumcols): log2 c steps u <- u + Rot(u, 2^(log2 c - 1 - t)),
    the binary first-column mask, then log2 c steps s <- s + Rot(s, -2^t);
  * RE-Matmul = sumrows(A_exp x W), CE-Matmul = sumcols(A_rep x W) (Sec. 4.2.1);
  * EncryptedPolyReLU A = Z x Z + Z (Sec. 4.2.2);
  * Alg. 1: forward, RSS gradient Yhat - Y, delta W_col = A_rep x grad,
    delta A = RE-Matmul(grad, W_col), delta Z = 1 + 2 x delta A (the paper's
    EncryptedPolyReLU' evaluated at delta A), delta W_row = A_exp x delta Z;
  * Alg. 2: decay, NAG velocity and update, then Bootstrap of W and V.
Readings of the design notes: R1 the 784 features are split into row tiles of
r and RE-Matmul sums the tile products before sumrows; R2 per-sample
gradients are added (+ of ciphertexts) over the mini-batch, 1/b folded into
gamma; R3 the local classifier's update uses the previous iteration's
gradient (Alg. 1) and, at the first iteration, the current one; R4 non-integer
constants multiply as round(c q_l S_target / S) followed by a rescale, so every
sum meets at one scale (an operand at a higher level is brought down the
same way); integer constants (the 2 of delta Z) cost no level (C14); R5
ciphertext products go through the bootstrapping evaluator's multiply, with
ModDown and rescale merged (C21).
`plain_step` is the same computation on FP64 slot vectors (numpy).

CE-Block (Sec. 4.2.3: the alternation of RE- and CE-Blocks; Sec. 4.3 notes
that the extension of Alg. 1 to CE-Blocks is straightforward) -- reading R6:
the dual of Alg. 1 with the formats swapped.  Input A_rep (a RE-Block's
activations); Z_exp = CE-Matmul(A_rep, W_col); A_exp = EncryptedPolyReLU(Z);
the local classifier is a RE-FC layer, Yhat_rep = RE-Matmul(A_exp, W_row*);
grad = Yhat - Y_rep; delta W_row* = A_exp x grad; delta A_exp =
CE-Matmul(grad, W_row*); delta Z = 1 + 2 delta A; delta W_col = A_rep x
delta Z; the same Alg. 2 updates and bootstraps (R2-R5 as for the RE-Block).
`plain_step_ce` is its FP64 slot form.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import OCt, Oracle
from .bootstrap import BootPlan, Evaluator, round_half_away


@dataclass(frozen=True)
class Geometry:
    r: int
    c: int
    k0: int
    k1: int
    o: int

    @property
    def tiles(self) -> int:
        return -(-self.k0 // self.r)

    def rotation_steps(self) -> list:
        lr, lc = int(math.log2(self.r)), int(math.log2(self.c))
        steps = [self.c * (1 << (lr - 1 - t)) for t in range(lr)]
        steps += [1 << (lc - 1 - t) for t in range(lc)]
        steps += [-(1 << t) for t in range(lc)]
        return steps


# ---------------------------------------------------------------- packing (Sec. 4.1)
def pack_expanded(vec, g: Geometry) -> np.ndarray:
    m = np.zeros((g.r, g.c))
    m[: len(vec), :] = np.asarray(vec)[:, None]
    return m.ravel()


def pack_repeated(vec, g: Geometry) -> np.ndarray:
    m = np.zeros((g.r, g.c))
    m[:, : len(vec)] = np.asarray(vec)[None, :]
    return m.ravel()


def pack_rowwise(w, g: Geometry) -> np.ndarray:
    m = np.zeros((g.r, g.c))
    m[: w.shape[0], : w.shape[1]] = w
    return m.ravel()


def pack_colwise(w, g: Geometry) -> np.ndarray:
    m = np.zeros((g.r, g.c))
    m[: w.shape[1], : w.shape[0]] = w.T
    return m.ravel()


def first_column_mask(g: Geometry) -> np.ndarray:
    m = np.zeros((g.r, g.c))
    m[:, 0] = 1.0
    return m.ravel()


def tile_inputs(x, g: Geometry) -> list:
    xp = np.zeros(g.tiles * g.r)
    xp[: len(x)] = x
    return [pack_expanded(xp[t * g.r:(t + 1) * g.r], g) for t in range(g.tiles)]


def tile_weights(w, g: Geometry) -> list:
    wp = np.zeros((g.tiles * g.r, w.shape[1]))
    wp[: w.shape[0]] = w
    return [pack_rowwise(wp[t * g.r:(t + 1) * g.r], g) for t in range(g.tiles)]


# ---------------------------------------------------------------- FP64 slot reference
def _rot(v, k):
    return np.roll(v, -k)


def plain_sumrows(v, g):
    for t in range(int(math.log2(g.r))):
        v = v + _rot(v, g.c * (1 << (int(math.log2(g.r)) - 1 - t)))
    return v


def plain_sumcols(v, g):
    lc = int(math.log2(g.c))
    for t in range(lc):
        v = v + _rot(v, 1 << (lc - 1 - t))
    v = v * first_column_mask(g)
    for t in range(lc):
        v = v + _rot(v, -(1 << t))
    return v


def plain_update(w, v, dw, gamma, eta, mu, first):
    dw = dw + eta * dw
    if first:
        v_new = dw
        delta = gamma * dw + gamma * mu * dw
    else:
        v_new = mu * v + dw
        delta = gamma * dw + gamma * mu * dw + gamma * mu * mu * v
    return w - delta, v_new


def plain_step(state, xs, ys, g: Geometry, gamma, eta, mu, first):
    """Slot vectors through Alg. 1 / Alg. 2 (no bootstrapping needed)."""
    W, V, Ws, Vs, dWs_prev = state
    dW = [np.zeros(g.r * g.c) for _ in range(g.tiles)]
    dWs = np.zeros(g.r * g.c)
    for x, y in zip(xs, ys):
        z = plain_sumrows(sum(x[t] * W[t] for t in range(g.tiles)), g)
        a = z * z + z
        yhat = plain_sumcols(a * Ws, g)
        grad = yhat - y
        dWs = dWs + a * grad
        da = plain_sumrows(grad * Ws, g)
        dz = 1 + 2 * da
        for t in range(g.tiles):
            dW[t] = dW[t] + x[t] * dz
    newW, newV = [], []
    for t in range(g.tiles):
        w1, v1 = plain_update(W[t], V[t], dW[t], gamma, eta, mu, first)
        newW.append(w1)
        newV.append(v1)
    grad_s = dWs if dWs_prev is None else dWs_prev
    ws1, vs1 = plain_update(Ws, Vs, grad_s, gamma, eta, mu, first)
    return newW, newV, ws1, vs1, dWs


def plain_step_ce(state, as_rep, ys_rep, g: Geometry, gamma, eta, mu, first):
    """CE-Block (reading R6) on FP64 slot vectors; also returns A_exp per sample."""
    W, V, Ws, Vs, dWs_prev = state
    dW = np.zeros(g.r * g.c)
    dWs = np.zeros(g.r * g.c)
    acts = []
    for a, y in zip(as_rep, ys_rep):
        z = plain_sumcols(a * W, g)
        act = z * z + z
        acts.append(act)
        yhat = plain_sumrows(act * Ws, g)
        grad = yhat - y
        dWs = dWs + act * grad
        da = plain_sumcols(grad * Ws, g)
        dz = 1 + 2 * da
        dW = dW + a * dz
    w1, v1 = plain_update(W, V, dW, gamma, eta, mu, first)
    grad_s = dWs if dWs_prev is None else dWs_prev
    ws1, vs1 = plain_update(Ws, Vs, grad_s, gamma, eta, mu, first)
    return (w1, v1, ws1, vs1, dWs), acts


# ---------------------------------------------------------------- encrypted step
class REBlock:
    """Alg. 1 + Alg. 2 for one RE-Block over the oracle's primitives."""

    def __init__(self, orc: Oracle, g: Geometry, gamma, eta, mu, boot: Evaluator | None = None,
                 mask_coeffs=None):
        self.o = orc
        self.g = g
        self.gamma, self.eta, self.mu = gamma, eta, mu
        self.boot = boot
        self.ev = boot if boot is not None else Evaluator.__new__(Evaluator)
        self.ev.o = orc
        self._mask = mask_coeffs  # integer plaintext of the mask (None: encode here)

    # ---- helpers shared with the bootstrapping evaluator's scale rules
    def mul(self, a: OCt, b: OCt) -> OCt:
        return Evaluator.mul(self.ev, a, b)

    def add(self, a, b):
        return Evaluator.add(self.ev, a, b)

    def sub(self, a, b):
        return Evaluator.sub(self.ev, a, b)

    def mul_const(self, ct: OCt, cst: float, target_scale: float) -> OCt:
        ql = float(self.o.q[ct.level])
        k = round_half_away(cst * (ql * target_scale / ct.scale))
        r = self.o.mul_int(ct, k)
        r.scale = ql * target_scale
        return self.o.rescale(r)

    def add_const(self, ct: OCt, cst: float) -> OCt:
        return Evaluator.add_const(self.ev, ct, cst)

    def mask_mult(self, ct: OCt) -> OCt:
        ql = float(self.o.q[ct.level])
        if self._mask is None:
            m = self.o.encode(first_column_mask(self.g), ql)
        else:
            m = self._mask
        r = self.o.mul_plain(ct, self.o.pt_from_int(m, ct.level), ql)
        return self.o.rescale(r)

    def sumrows(self, ct):
        lr = int(math.log2(self.g.r))
        for t in range(lr):
            ct = self.o.add(ct, self.o.rotate(ct, self.g.c * (1 << (lr - 1 - t))))
        return ct

    def sumcols(self, ct):
        lc = int(math.log2(self.g.c))
        for t in range(lc):
            ct = self.o.add(ct, self.o.rotate(ct, 1 << (lc - 1 - t)))
        ct = self.mask_mult(ct)
        for t in range(lc):
            ct = self.o.add(ct, self.o.rotate(ct, -(1 << t)))
        return ct

    # ---- Alg. 2
    def update(self, w, v, dw, first):
        dw = self.add(dw, self.mul_const(dw, self.eta, dw.scale))
        s = dw.scale
        if first:
            v_new = dw
            delta = self.add(self.mul_const(dw, self.gamma, s), self.mul_const(dw, self.gamma * self.mu, s))
        else:
            v_new = self.add(self.mul_const(v, self.mu, s), dw)
            delta = self.add(self.mul_const(dw, self.gamma, s), self.mul_const(dw, self.gamma * self.mu, s))
            delta = self.add(delta, self.mul_const(v, self.gamma * self.mu * self.mu, s))
        return self.sub(w, delta), v_new

    # ---- Alg. 1
    def step(self, state, xs, ys, first: bool, bootstrap: bool = True):
        W, V, Ws, Vs, dWs_prev = state
        T = self.g.tiles
        dW = [None] * T
        dWs = None
        self.last_activations = []  # A_rep per sample: the next (CE-)Block's input
        for x, y in zip(xs, ys):
            acc = None
            for t in range(T):
                p = self.mul(x[t], W[t])
                acc = p if acc is None else self.o.add(acc, p)
            z = self.sumrows(acc)                                  # RE-Matmul
            a = self.add(self.mul(z, z), z)                        # EncryptedPolyReLU
            self.last_activations.append(a)
            yhat = self.sumcols(self.mul(a, Ws))                   # CE-Matmul
            grad = self.sub(yhat, y)                               # RSS gradient
            dws = self.mul(a, grad)                                # delta W_col
            da = self.sumrows(self.mul(grad, Ws))                  # RE-Matmul(grad, W_col)
            dz = self.add_const(self.o.mul_int(da, 2), 1.0)        # EncryptedPolyReLU'
            dWs = dws if dWs is None else self.o.add(dWs, dws)
            for t in range(T):
                d = self.mul(x[t], dz)                             # delta W_row
                dW[t] = d if dW[t] is None else self.o.add(dW[t], d)
        newW, newV = [], []
        for t in range(T):
            w1, v1 = self.update(W[t], V[t], dW[t], first)
            newW.append(w1)
            newV.append(v1)
        ws1, vs1 = self.update(Ws, Vs, dWs if dWs_prev is None else dWs_prev, first)
        if bootstrap:
            newW = [self.boot.bootstrap(c) for c in newW]
            newV = [self.boot.bootstrap(c) for c in newV]
            ws1 = self.boot.bootstrap(ws1)
            vs1 = self.boot.bootstrap(vs1)
        return newW, newV, ws1, vs1, dWs


class CEBlock(REBlock):
    """Reading R6: a CE-Block's step over the oracle's primitives (the dual of
    Alg. 1); W is the CE-FC layer's column-wise matrix, Ws the RE-FC local
    classifier's row-wise matrix."""

    def step(self, state, as_rep, ys, first: bool, bootstrap: bool = True):
        W, V, Ws, Vs, dWs_prev = state
        dW = dWs = None
        self.last_activations = []  # A_exp per sample
        for a, y in zip(as_rep, ys):
            z = self.sumcols(self.mul(a, W))                       # CE-Matmul
            act = self.add(self.mul(z, z), z)                      # EncryptedPolyReLU
            self.last_activations.append(act)
            yhat = self.sumrows(self.mul(act, Ws))                 # RE-Matmul (local classifier)
            grad = self.sub(yhat, y)                               # RSS gradient
            dws = self.mul(act, grad)                              # delta W_row*
            da = self.sumcols(self.mul(grad, Ws))                  # CE-Matmul(grad, W_row*)
            dz = self.add_const(self.o.mul_int(da, 2), 1.0)        # EncryptedPolyReLU'
            dw = self.mul(a, dz)                                   # delta W_col
            dWs = dws if dWs is None else self.o.add(dWs, dws)
            dW = dw if dW is None else self.o.add(dW, dw)
        w1, v1 = self.update(W, V, dW, first)
        ws1, vs1 = self.update(Ws, Vs, dWs if dWs_prev is None else dWs_prev, first)
        if bootstrap:
            w1, v1, ws1, vs1 = (self.boot.bootstrap(c) for c in (w1, v1, ws1, vs1))
        return w1, v1, ws1, vs1, dWs
