"""ReBoot RE-Block training step (Alg. 1 + Alg. 2) over the C ABI.

The encrypted forward pass, local-error backward pass, NAG update and
bootstrap of one RE-Block, batched across the mini-batch: every operation is
one batched library call over all samples (or over the block's weight
ciphertexts), so each kernel launch serves the whole batch.

CEBlock is the dual step of a CE-Block (reading R6: CE-Matmul forward, a
RE-FC local classifier, delta A by CE-Matmul), which takes a RE-Block's
activations; RE- and CE-Blocks alternate in eMLP-2/3 (Table 3).

Paper passages: packing (Sec. 4.1); sum across rows / columns (Sec. 3,
Eq. sumrows / sumcols); RE-Matmul and CE-Matmul (Sec. 4.2.1);
EncryptedPolyReLU A = Z x Z + Z (Sec. 4.2.2); Alg. 1 (forward, RSS gradient,
delta W_col, delta A, delta Z = 1 + 2 delta A, delta W_row, updates,
Bootstrap) and Alg. 2 (decay, NAG velocity and weight update).  Readings:
features in row tiles of r summed before sumrows; per-sample gradients added
over the batch (1/b folded into gamma); the local classifier uses the
previous iteration's gradient (the current one at the first iteration);
non-integer constants multiply as round(c q_l S_target / S) then rescale and
sums meet at one scale (a higher operand is brought down by an integer
multiply and a rescale); the integer 2 of delta Z costs no level.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def round_half_away(x: float) -> int:
    t = math.trunc(x)
    if abs(x - t) >= 0.5:
        t += 1 if x > 0 else -1
    return int(t)


@dataclass(frozen=True)
class Geometry:
    """Encoding dimensions r x c = N/2 and the block's layer sizes."""
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
        return ([self.c * (1 << (lr - 1 - t)) for t in range(lr)] + [1 << (lc - 1 - t) for t in range(lc)]
                + [-(1 << t) for t in range(lc)])


# ---- Sec. 4.1 packing (host side, before encryption) ----
def pack_expanded(vec, g: Geometry) -> np.ndarray:
    m = np.zeros((g.r, g.c))
    m[: len(vec), :] = np.asarray(vec)[:, None]
    return m.ravel()


def pack_colwise(w, g: Geometry) -> np.ndarray:
    m = np.zeros((g.r, g.c))
    m[: w.shape[1], : w.shape[0]] = w.T
    return m.ravel()


def input_tiles(x, g: Geometry) -> list:
    xp = np.zeros(g.tiles * g.r)
    xp[: len(x)] = x
    return [pack_expanded(xp[t * g.r:(t + 1) * g.r], g) for t in range(g.tiles)]


def weight_tiles(w, g: Geometry) -> list:
    wp = np.zeros((g.tiles * g.r, w.shape[1]))
    wp[: w.shape[0]] = w
    out = []
    for t in range(g.tiles):
        m = np.zeros((g.r, g.c))
        m[:, : w.shape[1]] = wp[t * g.r:(t + 1) * g.r]
        out.append(m.ravel())
    return out


def first_column_mask(g: Geometry) -> np.ndarray:
    m = np.zeros((g.r, g.c))
    m[:, 0] = 1.0
    return m.ravel()


class REBlock:
    """One RE-Block on a bootstrapping-capable context (keys: relinearisation,
    conjugation, bootstrapping rotations and Geometry.rotation_steps())."""

    def __init__(self, ctx, g: Geometry, gamma: float, eta: float, mu: float, mask_coeffs=None,
                 iterative_log2_k: int | None = None):
        self.ctx = ctx
        self.g = g
        self.gamma, self.eta, self.mu = gamma, eta, mu
        self._mask_coeffs = mask_coeffs
        self._mask_pt = {}
        # None: one bootstrap per weight ciphertext (reading C16); k: the
        # two-pass iterative bootstrap with 2^k (reading B12), the other
        # reading of the step's two bootstrapping passes (Sec. 4.3.4)
        self.iterative_log2_k = iterative_log2_k

    def refresh(self, cts):
        """Bootstrap the block's updated weights and velocities."""
        if self.iterative_log2_k is None:
            return self.ctx.bootstrap_batch(cts)
        # the iterative batch takes one input scale: one call per scale
        groups = {}
        for i, c in enumerate(cts):
            groups.setdefault(c.scale, []).append(i)
        out = [None] * len(cts)
        for idx in groups.values():
            for i, r in zip(idx, self.ctx.bootstrap_iterative_batch([cts[i] for i in idx], self.iterative_log2_k)):
                out[i] = r
        return out

    # ---- list helpers: every list shares one level and one scale ----
    @staticmethod
    def _lvl(xs):
        lv = xs[0].level
        assert all(x.level == lv for x in xs)
        return lv

    def view(self, xs, level):
        from . import Ciphertext
        return [x if x.level == level else Ciphertext(x.data, level, x.scale) for x in xs]

    def mul(self, a, b):
        """Products at the lower level; ModDown and rescale merged (C21), as the
        bootstrapping evaluator multiplies."""
        from . import RESCALE_MERGED
        lv = min(self._lvl(a), self._lvl(b))
        out = [self.ctx.new_ct(lv + 1) for _ in a]
        self.ctx.mul_relin_batch(self.view(a, lv), self.view(b, lv), out, rescale=RESCALE_MERGED)
        return out

    def rescale(self, xs, scale):
        for x in xs:
            x.scale = scale
        self.ctx.rescale_batch(xs)
        return xs

    def align(self, xs, level, scale):
        lv = self._lvl(xs)
        if lv > level:
            ql = float(self.ctx.q[lv])
            k = round_half_away(scale * ql / xs[0].scale)
            r = self.ctx.mul_int_batch(xs, k)
            r = self.rescale(r, scale * ql)
            return self.view(r, level)
        return self.view(xs, level)

    def _pair(self, a, b):
        la, lb = self._lvl(a), self._lvl(b)
        if la > lb:
            return self.align(a, lb, b[0].scale), b, b[0].scale
        if lb > la:
            return a, self.align(b, la, a[0].scale), a[0].scale
        return a, b, a[0].scale

    def add(self, a, b, subtract=False):
        x, y, s = self._pair(a, b)
        out = self.ctx.add_batch(x, y, subtract=subtract)
        for o in out:
            o.scale = s
        return out

    def plain_add(self, a, b):  # same level and scale: the library's own add
        return self.ctx.add_batch(a, b)

    def mul_const(self, xs, cst, target_scale):
        lv = self._lvl(xs)
        ql = float(self.ctx.q[lv])
        k = round_half_away(cst * (ql * target_scale / xs[0].scale))
        r = self.ctx.mul_int_batch(xs, k)
        return self.rescale(r, ql * target_scale)

    def add_const(self, xs, cst):
        lv = self._lvl(xs)
        m = np.zeros(self.ctx.n, dtype=np.int64)
        m[0] = round_half_away(cst * xs[0].scale)
        return self.ctx.add_plain_batch(xs, self.ctx.pt_from_int(m, lv))

    def mask_mult(self, xs):
        lv = self._lvl(xs)
        ql = float(self.ctx.q[lv])
        if lv not in self._mask_pt:
            if self._mask_coeffs is None:
                self._mask_pt[lv] = self.ctx.encode(first_column_mask(self.g), lv, ql)
            else:
                self._mask_pt[lv] = self.ctx.pt_from_int(self._mask_coeffs[lv], lv)
        r = self.ctx.mul_plain_batch(xs, self._mask_pt[lv], ql)
        self.ctx.rescale_batch(r)
        return r

    def rotate(self, xs, k):
        out = [self.ctx.new_ct(x.level + 1) for x in xs]
        self.ctx.rotate_batch(xs, [k] * len(xs), out)
        return out

    def sumrows(self, xs):  # Eq. sumrows
        lr = int(math.log2(self.g.r))
        for t in range(lr):
            xs = self.plain_add(xs, self.rotate(xs, self.g.c * (1 << (lr - 1 - t))))
        return xs

    def sumcols(self, xs):  # Eq. sumcols
        lc = int(math.log2(self.g.c))
        for t in range(lc):
            xs = self.plain_add(xs, self.rotate(xs, 1 << (lc - 1 - t)))
        xs = self.mask_mult(xs)
        for t in range(lc):
            xs = self.plain_add(xs, self.rotate(xs, -(1 << t)))
        return xs

    # ---- Alg. 2 ----
    def update(self, w, v, dw, first):
        dw = self.add(dw, self.mul_const(dw, self.eta, dw[0].scale))
        s = dw[0].scale
        if first:
            v_new = dw
            delta = self.add(self.mul_const(dw, self.gamma, s), self.mul_const(dw, self.gamma * self.mu, s))
        else:
            v_new = self.add(self.mul_const(v, self.mu, s), dw)
            delta = self.add(self.mul_const(dw, self.gamma, s), self.mul_const(dw, self.gamma * self.mu, s))
            delta = self.add(delta, self.mul_const(v, self.gamma * self.mu * self.mu, s))
        return self.add(w, delta, subtract=True), v_new

    # ---- Alg. 1 ----
    def step(self, state, xs, ys, first: bool, bootstrap: bool = True):
        """state = (W tiles, V tiles, W*, V*, previous delta W* or None);
        xs[s][t]: input tile t of sample s; ys[s]: label of sample s."""
        W, V, Ws, Vs, dWs_prev = state
        T, S = self.g.tiles, len(xs)
        acc = None
        for t in range(T):
            p = self.mul([xs[s][t] for s in range(S)], [W[t]] * S)
            acc = p if acc is None else self.plain_add(acc, p)
        z = self.sumrows(acc)                                         # RE-Matmul
        a = self.add(self.mul(z, z), z)                               # EncryptedPolyReLU
        self.last_activations = a                                     # A_rep: a CE-Block's input
        yhat = self.sumcols(self.mul(a, [Ws] * S))                    # CE-Matmul
        grad = self.add(yhat, ys, subtract=True)                      # RSS gradient
        dws = self.mul(a, grad)                                       # delta W_col per sample
        da = self.sumrows(self.mul(grad, [Ws] * S))                   # RE-Matmul(grad, W_col)
        dz = self.add_const(self.ctx.mul_int_batch(da, 2), 1.0)       # EncryptedPolyReLU'
        dW = []
        for t in range(T):                                            # delta W_row per sample
            d = self.mul([xs[s][t] for s in range(S)], dz)
            total = [d[0]]
            for s in range(1, S):
                total = self.plain_add(total, [d[s]])
            dW.append(total[0])
        dWs = [dws[0]]
        for s in range(1, S):
            dWs = self.plain_add(dWs, [dws[s]])
        dWs = dWs[0]
        nw, nv = self.update(W, V, dW, first)
        grad_s = dWs if dWs_prev is None else dWs_prev
        ws1, vs1 = self.update([Ws], [Vs], [grad_s], first)
        new = (nw, nv, ws1[0], vs1[0], dWs)
        if not bootstrap:
            return new
        refreshed = self.refresh(nw + nv + ws1 + vs1)
        return refreshed[:T], refreshed[T:2 * T], refreshed[2 * T], refreshed[2 * T + 1], dWs


def pack_repeated(vec, g: Geometry) -> np.ndarray:
    m = np.zeros((g.r, g.c))
    m[:, : len(vec)] = np.asarray(vec)[None, :]
    return m.ravel()


def pack_rowwise(w, g: Geometry) -> np.ndarray:
    m = np.zeros((g.r, g.c))
    m[: w.shape[0], : w.shape[1]] = w
    return m.ravel()


class CEBlock(REBlock):
    """One CE-Block (reading R6): W is the CE-FC layer's column-wise matrix
    and Ws the RE-FC local classifier's row-wise matrix; the inputs are a
    RE-Block's activations A_rep, the labels are in the repeated format."""

    def step(self, state, as_rep, ys, first: bool, bootstrap: bool = True):
        W, V, Ws, Vs, dWs_prev = state
        S = len(as_rep)
        z = self.sumcols(self.mul(as_rep, [W] * S))                   # CE-Matmul
        a = self.add(self.mul(z, z), z)                               # EncryptedPolyReLU
        self.last_activations = a                                     # A_exp
        yhat = self.sumrows(self.mul(a, [Ws] * S))                    # RE-Matmul (local classifier)
        grad = self.add(yhat, ys, subtract=True)                      # RSS gradient
        dws = self.mul(a, grad)                                       # delta W_row* per sample
        da = self.sumcols(self.mul(grad, [Ws] * S))                   # CE-Matmul(grad, W_row*)
        dz = self.add_const(self.ctx.mul_int_batch(da, 2), 1.0)       # EncryptedPolyReLU'
        dw = self.mul(as_rep, dz)                                     # delta W_col per sample
        dW, dWs = [dw[0]], [dws[0]]
        for s in range(1, S):
            dW = self.plain_add(dW, [dw[s]])
            dWs = self.plain_add(dWs, [dws[s]])
        nw, nv = self.update([W], [V], dW, first)
        grad_s = dWs if dWs_prev is None else [dWs_prev]
        ws1, vs1 = self.update([Ws], [Vs], grad_s, first)
        if not bootstrap:
            return nw[0], nv[0], ws1[0], vs1[0], dWs[0]
        refreshed = self.refresh(nw + nv + ws1 + vs1)
        return refreshed[0], refreshed[1], refreshed[2], refreshed[3], dWs[0]
