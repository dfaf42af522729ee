"""Pins for the oracle's ReBoot RE-Block step: the packed slot computation
against the matrix formulas it stands for (Sec. 4.1-4.3), the multiplicative
depth against Table 1 / Table 3 (tau_ReBoot = 8 for one hidden layer), and the
encrypted step against the FP64 slot computation."""
import numpy as np
import pytest

import oracle
import oracle.bootstrap as ob
import oracle.reboot as rb
import synthetic_inputs as si

G = rb.Geometry(r=32, c=64, k0=60, k1=64, o=10)


def _data(seed, b):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, size=(b, G.k0))
    y = np.eye(G.o)[rng.integers(0, G.o, size=b)]
    w = rng.normal(0, 1 / np.sqrt(G.k0), size=(G.k0, G.k1))
    ws = rng.normal(0, 1 / np.sqrt(G.k1), size=(G.k1, G.o))
    return x, y, w, ws


def _unpack(v, g):
    return v.reshape(g.r, g.c)


def test_sums_and_matmuls_match_matrix_products():
    x, y, w, ws = _data(1, 1)
    # RE-Matmul: Z_rep = sumrows(A_exp * W_row) holds x W in every row
    z = rb.plain_sumrows(sum(a * b for a, b in zip(rb.tile_inputs(x[0], G), rb.tile_weights(w, G))), G)
    zm = _unpack(z, G)
    assert np.allclose(zm, np.tile(x[0] @ w, (G.r, 1)))
    # CE-Matmul: Yhat_exp = sumcols(A_rep * W_col) holds a W* in the first o rows, replicated
    a = x[0, : G.k1] if G.k0 >= G.k1 else np.pad(x[0], (0, G.k1 - G.k0))
    yh = _unpack(rb.plain_sumcols(rb.pack_repeated(a, G) * rb.pack_colwise(ws, G), G), G)
    assert np.allclose(yh[: G.o], np.tile((a @ ws)[:, None], (1, G.c)))
    assert np.allclose(yh[G.o:], 0)


def test_plain_step_is_alg1_alg2_in_matrix_form():
    x, y, w, ws = _data(2, 3)
    gamma, eta, mu = 0.01, 0.001, 0.9
    W = rb.tile_weights(w, G)
    V = [np.zeros_like(t) for t in W]
    Ws = rb.pack_colwise(ws, G)
    Vs = np.zeros_like(Ws)
    xs = [rb.tile_inputs(xi, G) for xi in x]
    ys = [rb.pack_expanded(yi, G) for yi in y]
    newW, newV, ws1, vs1, dws = rb.plain_step((W, V, Ws, Vs, None), xs, ys, G, gamma, eta, mu, first=True)
    # the same algorithm written with matrices
    dW = np.zeros_like(w)
    dWs = np.zeros_like(ws)
    for xi, yi in zip(x, y):
        z = xi @ w
        a = z * z + z
        yhat = a @ ws
        g = yhat - yi
        dWs += np.outer(a, g)
        da = ws @ g
        dz = 1 + 2 * da
        dW += np.outer(xi, dz)
    def upd(wm, dwm):
        dwm = dwm + eta * dwm
        return wm - (gamma * dwm + gamma * mu * dwm), dwm
    w1, v1 = upd(w, dW)
    ws1m, vs1m = upd(ws, dWs)
    got_w = np.concatenate([_unpack(t, G) for t in newW])[: G.k0, : G.k1]
    assert np.allclose(got_w, w1)
    assert np.allclose(_unpack(ws1, G)[: G.o, : G.k1], ws1m.T)
    assert np.allclose(_unpack(vs1, G)[: G.o, : G.k1], vs1m.T)


def test_depth_matches_table_1_and_3():
    # Table 1, ReBoot, H = 1: fw = floor(2.5) + floor(1.5 + 1) = 4, bw = floor(4.5 + 1 - 1) = 4
    H = 1
    tau = int(np.floor(2.5 * H)) + int(np.floor(1.5 + H % 2)) + int(np.floor(4.5 + 1 - H % 2))
    assert tau == 8
    # Table 3: l = 24 = tau_ReBoot + tau_bs with tau_bs = 16 (eMLP-1)
    assert len(si.BOOT_Q_BITS) - 1 == tau + 16


@pytest.fixture(scope="module")
def env():
    w = si.BOOT_SMALL
    plan = ob.make_plan(w.log_n, len(w.q_bits))
    o = oracle.Oracle(w.log_n, w.q_bits, w.p_bits, w.dnum, w.h, w.sigma)
    o.keygen(1)
    o.gen_rotation_keys(sorted(set(plan.rotation_steps()) | set(G.rotation_steps())))
    o.gen_galois_key(o.conj_elt())
    boot = ob.Evaluator(o, plan, ob.encode_constants(o, plan))
    return w, o, boot


def _encrypt_state(o, g, w, ws, level, scale, seed0):
    W = [o.encrypt(o.pt_from_int(o.encode(t, scale), level), level, scale, seed0 + i)
         for i, t in enumerate(rb.tile_weights(w, g))]
    V = [o.encrypt(o.pt_from_int(o.encode(np.zeros(g.r * g.c), scale), level), level, scale, seed0 + 50 + i)
         for i in range(g.tiles)]
    Ws = o.encrypt(o.pt_from_int(o.encode(rb.pack_colwise(ws, g), scale), level), level, scale, seed0 + 90)
    Vs = o.encrypt(o.pt_from_int(o.encode(np.zeros(g.r * g.c), scale), level), level, scale, seed0 + 91)
    return W, V, Ws, Vs


def test_encrypted_step_matches_fp64_and_uses_eight_levels(env):
    w_, o, boot = env
    x, y, w, ws = _data(3, 2)
    scale = 2.0 ** w_.log2_scale
    lvl = 8
    gamma, eta, mu = 0.01, 0.001, 0.9
    W, V, Ws, Vs = _encrypt_state(o, G, w, ws, lvl, scale, 100)
    xs = [[o.encrypt(o.pt_from_int(o.encode(t, scale), lvl), lvl, scale, 300 + 10 * s + i)
           for i, t in enumerate(rb.tile_inputs(x[s], G))] for s in range(len(x))]
    ys = [o.encrypt(o.pt_from_int(o.encode(rb.pack_expanded(y[s], G), scale), lvl), lvl, scale, 400 + s)
          for s in range(len(y))]
    blk = rb.REBlock(o, G, gamma, eta, mu, boot)
    newW, newV, ws1, vs1, dws = blk.step((W, V, Ws, Vs, None), xs, ys, first=True, bootstrap=False)
    assert all(c.level == 0 for c in newW)  # eight levels from level 8: tau_ReBoot = 8
    pW = rb.tile_weights(w, G)
    ref = rb.plain_step((pW, [np.zeros_like(t) for t in pW], rb.pack_colwise(ws, G), np.zeros(G.r * G.c), None),
                        [rb.tile_inputs(xi, G) for xi in x], [rb.pack_expanded(yi, G) for yi in y], G,
                        gamma, eta, mu, first=True)
    for ct, want in zip(newW + [ws1], ref[0] + [ref[2]]):
        assert np.max(np.abs(o.decrypt_decode(ct).real - want)) < 2.0 ** -16
    # bootstrapping the updated weights refreshes them to level 8 within 2^-12
    refreshed = boot.bootstrap(newW[0])
    assert refreshed.level == 8
    assert np.max(np.abs(o.decrypt_decode(refreshed).real - ref[0][0])) < 2.0 ** -12


# ---------------------------------------------------------------- CE-Block (reading R6)
GC = rb.Geometry(r=32, c=64, k0=48, k1=24, o=10)  # CE-FC 48 -> 24, RE-FC classifier 24 -> 10


def _data_ce(seed, b):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, size=(b, GC.k0))       # the previous RE-Block's activations
    y = np.eye(GC.o)[rng.integers(0, GC.o, size=b)]
    w = rng.normal(0, 1 / np.sqrt(GC.k0), size=(GC.k0, GC.k1))
    ws = rng.normal(0, 1 / np.sqrt(GC.k1), size=(GC.k1, GC.o))
    return a, y, w, ws


def test_plain_ce_step_is_the_dual_of_alg1_in_matrix_form():
    a, y, w, ws = _data_ce(5, 3)
    gamma, eta, mu = 0.01, 0.001, 0.9
    W, Ws = rb.pack_colwise(w, GC), rb.pack_rowwise(ws, GC)
    state = (W, np.zeros_like(W), Ws, np.zeros_like(Ws), None)
    (w1p, v1p, ws1p, vs1p, _), acts = rb.plain_step_ce(
        state, [rb.pack_repeated(ai, GC) for ai in a], [rb.pack_repeated(yi, GC) for yi in y], GC,
        gamma, eta, mu, first=True)
    dW = np.zeros_like(w)
    dWs = np.zeros_like(ws)
    for s, (ai, yi) in enumerate(zip(a, y)):
        z = ai @ w
        act = z * z + z
        assert np.allclose(_unpack(acts[s], GC)[: GC.k1], np.tile(act[:, None], (1, GC.c)))  # expanded
        g = act @ ws - yi
        dWs += np.outer(act, g)
        dz = 1 + 2 * (ws @ g)
        dW += np.outer(ai, dz)
    def upd(wm, dwm):
        dwm = dwm + eta * dwm
        return wm - (gamma * dwm + gamma * mu * dwm), dwm
    w1, v1 = upd(w, dW)
    ws1, vs1 = upd(ws, dWs)
    assert np.allclose(_unpack(w1p, GC)[: GC.k1, : GC.k0], w1.T)
    assert np.allclose(_unpack(v1p, GC)[: GC.k1, : GC.k0], v1.T)
    assert np.allclose(_unpack(ws1p, GC)[: GC.k1, : GC.o], ws1)
    assert np.allclose(_unpack(vs1p, GC)[: GC.k1, : GC.o], vs1)


def test_encrypted_ce_step_matches_fp64_within_eleven_levels(env):
    """A CE-Block fed at level 9 (a RE-Block's activations from level-11
    inputs) with weights at level 11 ends at level 0: Table 3's
    tau_ReBoot = 11 for eMLP-2's two blocks."""
    w_, o, boot = env
    a, y, w, ws = _data_ce(6, 2)
    scale = 2.0 ** w_.log2_scale
    gamma, eta, mu = 0.01, 0.001, 0.9
    enc = lambda v, lv, sd: o.encrypt(o.pt_from_int(o.encode(v, scale), lv), lv, scale, sd)  # noqa: E731
    W, Ws = enc(rb.pack_colwise(w, GC), 11, 700), enc(rb.pack_rowwise(ws, GC), 11, 701)
    V, Vs = enc(np.zeros(GC.r * GC.c), 11, 702), enc(np.zeros(GC.r * GC.c), 11, 703)
    acts = [enc(rb.pack_repeated(a[s], GC), 9, 710 + s) for s in range(len(a))]
    ys = [enc(rb.pack_repeated(y[s], GC), 9, 720 + s) for s in range(len(y))]
    blk = rb.CEBlock(o, GC, gamma, eta, mu, boot)
    w1, v1, ws1, vs1, dws = blk.step((W, V, Ws, Vs, None), acts, ys, first=True, bootstrap=False)
    assert w1.level == 0
    (pw, pv, pws, pvs, _), pacts = rb.plain_step_ce(
        (rb.pack_colwise(w, GC), np.zeros(GC.r * GC.c), rb.pack_rowwise(ws, GC), np.zeros(GC.r * GC.c), None),
        [rb.pack_repeated(ai, GC) for ai in a], [rb.pack_repeated(yi, GC) for yi in y], GC,
        gamma, eta, mu, first=True)
    for ct, want in ((w1, pw), (ws1, pws), (blk.last_activations[0], pacts[0])):
        assert np.max(np.abs(o.decrypt_decode(ct).real - want)) < 2.0 ** -16
