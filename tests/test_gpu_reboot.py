"""ReBoot RE-Block step on the GPU against the oracle (bit-exact limbs on a
small ring, without the bootstrap whose own parity is tested separately)
and against the FP64 slot computation at the config-3 size (N = 2^16,
r x c = 256 x 128, 784 -> 128 -> 10) including the bootstrap of the weights."""
import numpy as np
import pytest

import synthetic_inputs as si

pytestmark = pytest.mark.gpu


def _data(seed, b, k0, k1, o, x_hi=1.0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, x_hi, size=(b, k0))
    y = np.eye(o)[rng.integers(0, o, size=b)]
    w = rng.normal(0, 1 / np.sqrt(k0), size=(k0, k1))
    ws = rng.normal(0, 1 / np.sqrt(k1), size=(k1, o))
    return x, y, w, ws


@pytest.mark.parametrize("tensor_form", ["uint64", "tensor", "fused"])
def test_reboot_step_bit_exact_small_ring(tensor_form):
    import torch
    import oracle
    import oracle.bootstrap as ob
    import oracle.reboot as orb
    import paper_2506_19693_gb300 as ck
    import paper_2506_19693_gb300.reboot as rb
    torch.cuda.set_device(0)
    w_ = si.BOOT_SMALL
    g = rb.Geometry(32, 64, 60, 64, 10)
    go = orb.Geometry(32, 64, 60, 64, 10)
    ctx = ck.Context.from_workload(w_)
    ctx.set_form(tensor_form)
    try:
        ctx.keygen(1, rot_steps=g.rotation_steps())
        o = oracle.Oracle(w_.log_n, w_.q_bits, w_.p_bits, w_.dnum, w_.h, w_.sigma)
        o.keygen(1)
        o.gen_rotation_keys(go.rotation_steps())
        x, y, w, ws = _data(5, 2, g.k0, g.k1, g.o)
        scale, lvl = 2.0 ** w_.log2_scale, 8
        gamma, eta, mu = 0.01, 0.001, 0.9
        seed = [1000]

        def both(vec):
            m = o.encode(vec, scale)
            seed[0] += 1
            return (ctx.encrypt(ctx.pt_from_int(m, lvl), lvl, scale, seed[0]),
                    o.encrypt(o.pt_from_int(m, lvl), lvl, scale, seed[0]))

        Wp = [both(t) for t in orb.tile_weights(w, go)]
        Vp = [both(np.full(g.r * g.c, 0.01)) for _ in range(g.tiles)]
        Wsp = both(orb.pack_colwise(ws, go))
        Vsp = both(np.full(g.r * g.c, 0.02))
        xsp = [[both(t) for t in orb.tile_inputs(xi, go)] for xi in x]
        ysp = [both(orb.pack_expanded(yi, go)) for yi in y]
        mask = {l: o.encode(orb.first_column_mask(go), float(o.q[l])) for l in range(lvl + 1)}
        gpu = rb.REBlock(ctx, g, gamma, eta, mu, mask_coeffs=mask)
        orc = orb.REBlock(o, go, gamma, eta, mu, mask_coeffs=None)
        orc._mask = None
        # the oracle encodes the same mask itself at each level (same function, same integers)
        for first in (True, False):
            st_g = ([p[0] for p in Wp], [p[0] for p in Vp], Wsp[0], Vsp[0], None)
            st_o = ([p[1] for p in Wp], [p[1] for p in Vp], Wsp[1], Vsp[1], None)
            rg = gpu.step(st_g, [[p[0] for p in s] for s in xsp], [p[0] for p in ysp], first, bootstrap=False)
            ro = orc.step(st_o, [[p[1] for p in s] for s in xsp], [p[1] for p in ysp], first, bootstrap=False)
            for cg, co in zip(rg[0] + rg[1] + [rg[2], rg[3], rg[4]], ro[0] + ro[1] + [ro[2], ro[3], ro[4]]):
                assert (cg.level, cg.scale) == (co.level, co.scale)
                assert np.array_equal(ctx.export_ct(cg), co.data)
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_reboot_step_config3_size_with_bootstrap():
    import torch
    import oracle.reboot as orb
    import paper_2506_19693_gb300 as ck
    import paper_2506_19693_gb300.reboot as rb
    torch.cuda.set_device(0)
    w_ = si.BOOT
    g = rb.Geometry(256, 128, 784, 128, 10)
    go = orb.Geometry(256, 128, 784, 128, 10)
    ctx = ck.Context.from_workload(w_)
    try:
        ctx.keygen_boot(1, rot_steps=g.rotation_steps())
        ctx.boot_setup()
        x, y, w, ws = _data(6, 4, g.k0, g.k1, g.o)
        scale, lvl = 2.0 ** w_.log2_scale, 8
        gamma, eta, mu = 0.001 / 4, 0.001, 0.9
        seeds = iter(range(5000, 6000))
        enc = lambda v: ctx.encrypt(ctx.encode(v, lvl, scale), lvl, scale, next(seeds))  # noqa: E731
        W = [enc(t) for t in rb.weight_tiles(w, g)]
        V = [enc(np.zeros(g.r * g.c)) for _ in range(g.tiles)]
        Ws, Vs = enc(rb.pack_colwise(ws, g)), enc(np.zeros(g.r * g.c))
        xs = [[enc(t) for t in rb.input_tiles(xi, g)] for xi in x]
        ys = [enc(rb.pack_expanded(yi, g)) for yi in y]
        blk = rb.REBlock(ctx, g, gamma, eta, mu)
        nw, nv, ws1, vs1, dws = blk.step((W, V, Ws, Vs, None), xs, ys, first=True, bootstrap=True)
        assert all(c.level == len(w_.q_bits) - 17 for c in nw + nv + [ws1, vs1])
        pW = orb.tile_weights(w, go)
        ref = orb.plain_step((pW, [np.zeros_like(t) for t in pW], orb.pack_colwise(ws, go),
                              np.zeros(g.r * g.c), None),
                             [orb.tile_inputs(xi, go) for xi in x], [orb.pack_expanded(yi, go) for yi in y], go,
                             gamma, eta, mu, first=True)
        for ct, want in zip(nw + [ws1], ref[0] + [ref[2]]):
            assert np.max(np.abs(ctx.decrypt_decode(ct).real - want)) < 2.0 ** -12
    finally:
        ctx.close()


@pytest.mark.parametrize("tensor_form", ["uint64", "tensor", "fused"])
def test_ce_block_step_bit_exact_small_ring(tensor_form):
    """Reading R6: the CE-Block step (inputs at level 9 as a RE-Block leaves
    them, weights at level 11) equals the oracle's limb for limb."""
    import torch
    import oracle
    import oracle.reboot as orb
    import paper_2506_19693_gb300 as ck
    import paper_2506_19693_gb300.reboot as rb
    torch.cuda.set_device(0)
    w_ = si.BOOT_SMALL
    g = rb.Geometry(32, 64, 48, 24, 10)
    go = orb.Geometry(32, 64, 48, 24, 10)
    ctx = ck.Context.from_workload(w_)
    ctx.set_form(tensor_form)
    try:
        ctx.keygen(1, rot_steps=g.rotation_steps())
        o = oracle.Oracle(w_.log_n, w_.q_bits, w_.p_bits, w_.dnum, w_.h, w_.sigma)
        o.keygen(1)
        o.gen_rotation_keys(go.rotation_steps())
        a, y, w, ws = _data(6, 2, g.k0, g.k1, g.o)
        scale = 2.0 ** w_.log2_scale
        gamma, eta, mu = 0.01, 0.001, 0.9
        seed = [2000]

        def both(vec, lvl):
            m = o.encode(vec, scale)
            seed[0] += 1
            return (ctx.encrypt(ctx.pt_from_int(m, lvl), lvl, scale, seed[0]),
                    o.encrypt(o.pt_from_int(m, lvl), lvl, scale, seed[0]))

        Wp, Wsp = both(orb.pack_colwise(w, go), 11), both(orb.pack_rowwise(ws, go), 11)
        Vp, Vsp = both(np.full(g.r * g.c, 0.01), 11), both(np.full(g.r * g.c, 0.02), 11)
        asp = [both(orb.pack_repeated(ai, go), 9) for ai in a]
        ysp = [both(orb.pack_repeated(yi, go), 9) for yi in y]
        mask = {l: o.encode(orb.first_column_mask(go), float(o.q[l])) for l in range(12)}
        gpu = rb.CEBlock(ctx, g, gamma, eta, mu, mask_coeffs=mask)
        orc = orb.CEBlock(o, go, gamma, eta, mu)
        for first in (True, False):
            rg = gpu.step((Wp[0], Vp[0], Wsp[0], Vsp[0], None), [p[0] for p in asp], [p[0] for p in ysp], first,
                          bootstrap=False)
            ro = orc.step((Wp[1], Vp[1], Wsp[1], Vsp[1], None), [p[1] for p in asp], [p[1] for p in ysp], first,
                          bootstrap=False)
            assert rg[0].level == 0
            for cg, co in zip(list(rg) + gpu.last_activations, list(ro) + orc.last_activations):
                assert (cg.level, cg.scale) == (co.level, co.scale)
                assert np.array_equal(ctx.export_ct(cg), co.data)
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_emlp2_step_at_2_17_matches_fp64():
    """eMLP-2 (Table 3: RE-Block(64) -> CE-Block(32), N = 2^17, l = 27): one
    step of both blocks, the CE-Block fed the RE-Block's activations, with the
    bootstraps; the refreshed weights decrypt to the FP64 slot computation."""
    import torch
    import oracle.reboot as orb
    import paper_2506_19693_gb300 as ck
    import paper_2506_19693_gb300.reboot as rb
    torch.cuda.set_device(0)
    wb = si.BOOT17
    g1, g2 = rb.Geometry(256, 256, 784, 64, 10), rb.Geometry(256, 256, 64, 32, 10)
    o1, o2 = orb.Geometry(256, 256, 784, 64, 10), orb.Geometry(256, 256, 64, 32, 10)
    ctx = ck.Context.from_workload(wb)
    try:
        ctx.keygen_boot(1)
        ctx.boot_setup()
        for k in sorted(set(g1.rotation_steps()) | set(g2.rotation_steps())):
            ctx.keygen_galois(ctx.galois_elt(k))
        b = 2
        rng = np.random.default_rng(31)
        x = rng.uniform(0, 1, size=(b, 784))
        y = np.eye(10)[rng.integers(0, 10, size=b)]
        w1 = rng.normal(0, 1 / np.sqrt(784), size=(784, 64))
        ws1 = rng.normal(0, 1 / 8, size=(64, 10))
        w2 = rng.normal(0, 1 / 8, size=(64, 32))
        ws2 = rng.normal(0, 1 / np.sqrt(32), size=(32, 10))
        gamma, eta, mu = 0.01, 0.001, 0.9
        scale, lvl = 2.0 ** wb.log2_scale, len(wb.q_bits) - 17
        seeds = iter(range(5000, 9000))
        enc = lambda v: ctx.encrypt(ctx.encode(v, lvl, scale), lvl, scale, next(seeds))  # noqa: E731
        zero = np.zeros(g1.r * g1.c)
        W1p, Ws1p = orb.tile_weights(w1, o1), orb.pack_colwise(ws1, o1)
        W2p, Ws2p = orb.pack_colwise(w2, o2), orb.pack_rowwise(ws2, o2)
        st1 = ([enc(t) for t in W1p], [enc(zero) for _ in W1p], enc(Ws1p), enc(zero), None)
        st2 = (enc(W2p), enc(zero), enc(Ws2p), enc(zero), None)
        xp = [orb.tile_inputs(xi, o1) for xi in x]
        yexp = [orb.pack_expanded(yi, o1) for yi in y]
        yrep = [orb.pack_repeated(yi, o2) for yi in y]
        blk1 = rb.REBlock(ctx, g1, gamma, eta, mu)
        blk2 = rb.CEBlock(ctx, g2, gamma, eta, mu)
        r1 = blk1.step(st1, [[enc(t) for t in xs] for xs in xp], [enc(v) for v in yexp], True)
        r2 = blk2.step(st2, blk1.last_activations, [enc(v) for v in yrep], True)
        # FP64: the RE-Block, its activations, then the CE-Block on them
        p1 = orb.plain_step((W1p, [zero] * len(W1p), Ws1p, zero, None), xp, yexp, o1, gamma, eta, mu, True)
        acts = []
        for xs in xp:
            z = orb.plain_sumrows(sum(a * w for a, w in zip(xs, W1p)), o1)
            acts.append(z * z + z)
        p2, _ = orb.plain_step_ce((W2p, zero, Ws2p, zero, None), acts, yrep, o2, gamma, eta, mu, True)
        assert r1[0][0].level == r2[0].level == lvl
        for ct, want in ((r1[0][0], p1[0][0]), (r1[2], p1[2]), (r2[0], p2[0]), (r2[2], p2[2])):
            assert np.max(np.abs(ctx.decrypt_decode(ct).real - want)) < 2.0 ** -12
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_emlp3_step_at_2_17_matches_fp64():
    """eMLP-3 (Table 3: RE-Block(128) -> CE-Block(64) -> RE-Block(32), N = 2^17,
    l = 29 = 13 + 16): the third block is a RE-Block fed the CE-Block's
    activations as its single input tile; it ends exactly at level 0 before
    its bootstrap.  All refreshed weights decrypt to the FP64 computation."""
    import torch
    import oracle.reboot as orb
    import paper_2506_19693_gb300 as ck
    import paper_2506_19693_gb300.reboot as rb
    torch.cuda.set_device(0)
    wb = si.BOOT17_L29
    dims = [(784, 128), (128, 64), (64, 32)]
    gs = [rb.Geometry(256, 256, k0, k1, 10) for k0, k1 in dims]
    os_ = [orb.Geometry(256, 256, k0, k1, 10) for k0, k1 in dims]
    ctx = ck.Context.from_workload(wb)
    try:
        ctx.keygen_boot(1)
        ctx.boot_setup()
        for k in sorted(set(gs[0].rotation_steps())):
            ctx.keygen_galois(ctx.galois_elt(k))
        b = 2
        rng = np.random.default_rng(41)
        x = rng.uniform(0, 1, size=(b, 784))
        y = np.eye(10)[rng.integers(0, 10, size=b)]
        ws_ = [rng.normal(0, 1 / np.sqrt(k0), size=(k0, k1)) for k0, k1 in dims]
        cs_ = [rng.normal(0, 1 / np.sqrt(k1), size=(k1, 10)) for _, k1 in dims]
        gamma, eta, mu = 0.01, 0.001, 0.9
        scale, lvl = 2.0 ** wb.log2_scale, len(wb.q_bits) - 17
        assert lvl == 13
        seeds = iter(range(9000, 13000))
        enc = lambda v: ctx.encrypt(ctx.encode(v, lvl, scale), lvl, scale, next(seeds))  # noqa: E731
        zero = np.zeros(256 * 256)
        # block 1 (RE), block 2 (CE), block 3 (RE) in their packings
        P1 = (orb.tile_weights(ws_[0], os_[0]), orb.pack_colwise(cs_[0], os_[0]))
        P2 = (orb.pack_colwise(ws_[1], os_[1]), orb.pack_rowwise(cs_[1], os_[1]))
        P3 = (orb.tile_weights(ws_[2], os_[2]), orb.pack_colwise(cs_[2], os_[2]))
        st1 = ([enc(t) for t in P1[0]], [enc(zero) for _ in P1[0]], enc(P1[1]), enc(zero), None)
        st2 = (enc(P2[0]), enc(zero), enc(P2[1]), enc(zero), None)
        st3 = ([enc(t) for t in P3[0]], [enc(zero) for _ in P3[0]], enc(P3[1]), enc(zero), None)
        xp = [orb.tile_inputs(xi, os_[0]) for xi in x]
        yexp = [orb.pack_expanded(yi, os_[0]) for yi in y]
        yrep = [orb.pack_repeated(yi, os_[0]) for yi in y]
        b1, b2 = rb.REBlock(ctx, gs[0], gamma, eta, mu), rb.CEBlock(ctx, gs[1], gamma, eta, mu)
        b3 = rb.REBlock(ctx, gs[2], gamma, eta, mu)
        r1 = b1.step(st1, [[enc(t) for t in xs] for xs in xp], [enc(v) for v in yexp], True)
        r2 = b2.step(st2, b1.last_activations, [enc(v) for v in yrep], True)
        ye = [enc(v) for v in yexp]
        r3 = b3.step(st3, [[a] for a in b2.last_activations], ye, True, bootstrap=False)
        assert r3[0][0].level == 0  # tau_ReBoot = 13 used exactly
        r3 = b3.step(st3, [[a] for a in b2.last_activations], ye, True)
        # FP64
        p1 = orb.plain_step((P1[0], [zero] * len(P1[0]), P1[1], zero, None), xp, yexp, os_[0], gamma, eta, mu, True)
        a1 = []
        for xs in xp:
            z = orb.plain_sumrows(sum(u * w for u, w in zip(xs, P1[0])), os_[0])
            a1.append(z * z + z)
        p2, a2 = orb.plain_step_ce((P2[0], zero, P2[1], zero, None), a1, yrep, os_[1], gamma, eta, mu, True)
        p3 = orb.plain_step((P3[0], [zero] * len(P3[0]), P3[1], zero, None), [[a] for a in a2], yexp, os_[2],
                            gamma, eta, mu, True)
        for ct, want in ((r1[0][0], p1[0][0]), (r2[0], p2[0]), (r2[2], p2[2]), (r3[0][0], p3[0][0]),
                         (r3[2], p3[2])):
            assert ct.level == lvl
            assert np.max(np.abs(ctx.decrypt_decode(ct).real - want)) < 2.0 ** -12
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_reboot_step_with_iterative_bootstrap_is_more_precise():
    """The other reading of the step's two bootstrapping iterations (C16 / B12):
    with the two-pass bootstrap the refreshed weights are much closer to FP64."""
    import torch
    import oracle.reboot as orb
    import paper_2506_19693_gb300 as ck
    import paper_2506_19693_gb300.reboot as rb
    torch.cuda.set_device(0)
    wb = si.BOOT
    g, go = rb.Geometry(256, 128, 784, 128, 10), orb.Geometry(256, 128, 784, 128, 10)
    ctx = ck.Context.from_workload(wb)
    try:
        ctx.keygen_boot(1)
        ctx.boot_setup()
        for k in g.rotation_steps():
            ctx.keygen_galois(ctx.galois_elt(k))
        x, y, w, ws = _data(7, 2, g.k0, g.k1, g.o)
        gamma, eta, mu = 0.01, 0.001, 0.9
        scale, lvl = 2.0 ** wb.log2_scale, len(wb.q_bits) - 17
        seeds = iter(range(20000, 30000))
        enc = lambda v: ctx.encrypt(ctx.encode(v, lvl, scale), lvl, scale, next(seeds))  # noqa: E731
        Wp, Wsp = orb.tile_weights(w, go), orb.pack_colwise(ws, go)
        zero = np.zeros(g.r * g.c)
        xs = [[enc(t) for t in orb.tile_inputs(xi, go)] for xi in x]
        ys = [enc(orb.pack_expanded(yi, go)) for yi in y]
        ref = orb.plain_step((Wp, [zero] * len(Wp), Wsp, zero, None), [orb.tile_inputs(xi, go) for xi in x],
                             [orb.pack_expanded(yi, go) for yi in y], go, gamma, eta, mu, True)
        errs = {}
        for k in (None, 16):
            st = ([enc(t) for t in Wp], [enc(zero) for _ in Wp], enc(Wsp), enc(zero), None)
            r = rb.REBlock(ctx, g, gamma, eta, mu, iterative_log2_k=k).step(st, xs, ys, True)
            assert r[0][0].level == lvl
            errs[k] = max(np.max(np.abs(ctx.decrypt_decode(c).real - want))
                          for c, want in zip(r[0] + [r[2]], ref[0] + [ref[2]]))
        assert errs[None] < 2.0 ** -12 and errs[16] < 2.0 ** -26 and errs[16] < errs[None] / 64, errs
        assert ctx.device_error() == 0
    finally:
        ctx.close()


def test_reboot_trajectory_follows_fp64_simulator():
    """Five chained RE-Block steps (NAG with velocity after the first), a new
    two-sample mini-batch each step, W, V, W*, V* bootstrapped at the end of
    every step and fed to the next: after every step the decrypted weights stay
    within 2^-14 of the FP64 simulator carried along the same data.  Inputs in
    [0, 1/4] and gamma = 10^-3 keep the simulator's own trajectory bounded
    (|V| <= 2 over the five steps; at gamma = 0.05 it diverges in FP64 too)."""
    import torch
    import oracle.reboot as orb
    import paper_2506_19693_gb300 as ck
    import paper_2506_19693_gb300.reboot as rb
    torch.cuda.set_device(0)
    w_ = si.BOOT_SMALL
    g = rb.Geometry(32, 64, 60, 64, 10)
    go = orb.Geometry(32, 64, 60, 64, 10)
    ctx = ck.Context.from_workload(w_)
    try:
        ctx.keygen_boot(1, rot_steps=g.rotation_steps())
        ctx.boot_setup()
        _, _, w, ws = _data(9, 2, g.k0, g.k1, g.o)
        scale, lvl = 2.0 ** w_.log2_scale, len(w_.q_bits) - 17
        gamma, eta, mu = 0.001, 0.001, 0.9
        seeds = iter(range(7000, 9000))
        enc = lambda v: ctx.encrypt(ctx.encode(v, lvl, scale), lvl, scale, next(seeds))  # noqa: E731
        state = ([enc(t) for t in rb.weight_tiles(w, g)], [enc(np.zeros(g.r * g.c)) for _ in range(g.tiles)],
                 enc(rb.pack_colwise(ws, g)), enc(np.zeros(g.r * g.c)), None)
        pW = orb.tile_weights(w, go)
        ref = (pW, [np.zeros_like(t) for t in pW], orb.pack_colwise(ws, go), np.zeros(g.r * g.c), None)
        blk = rb.REBlock(ctx, g, gamma, eta, mu)
        errs = []
        for step in range(5):
            x, y, _, _ = _data(100 + step, 2, g.k0, g.k1, g.o, x_hi=0.25)
            xs = [[enc(t) for t in rb.input_tiles(xi, g)] for xi in x]
            ys = [enc(rb.pack_expanded(yi, g)) for yi in y]
            state = blk.step(state, xs, ys, first=step == 0, bootstrap=True)
            ref = orb.plain_step(ref, [orb.tile_inputs(xi, go) for xi in x],
                                 [orb.pack_expanded(yi, go) for yi in y], go, gamma, eta, mu, first=step == 0)
            got = state[0] + state[1] + [state[2], state[3]]
            want = ref[0] + ref[1] + [ref[2], ref[3]]
            errs.append(max(np.max(np.abs(ctx.decrypt_decode(c).real - v)) for c, v in zip(got, want)))
            assert all(c.level == lvl for c in got)
        assert max(errs) < 2.0 ** -14, errs
        # the weights moved: the trajectory is not the starting point
        assert np.max(np.abs(ref[0][0] - pW[0])) > 20 * max(errs)
        assert ctx.device_error() == 0
    finally:
        ctx.close()
