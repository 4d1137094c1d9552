"""GPU parity of the learned part: learned-model rANS decode (bit-exact against the oracle),
the library's learned encoder (bytes against the oracle), fp32 training kernels (against the
fp64 oracle to 1e-4 relative) and the learned model's gain over channel-wise coding."""
import numpy as np
import pytest

from oracle import model as M
from oracle import scene as S
from paper_2607_12656_b300 import sgs
from paper_2607_12656_b300.scenegen import kaiming_init, make_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_decode import gpu_decode, same_bits  # noqa: E402
from tolerance import assert_close  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = sgs.Context(0, 1 << 20)
    yield c
    c.close()


@pytest.fixture(scope="module")
def toy():
    sc = make_scene(3000, 21)
    P = S.prepare(sc.pos, sc.attr, 10, 8)
    q = P.q.astype(np.uint8)
    lr = S.lane_bounds(P.n_rows, 16)
    p, _ = M.train(kaiming_init(2), q, lr, 60, 2048, seed=4, lr=3e-3)
    model = M.freeze({k: v.astype(np.float32) for k, v in p.items()}, q, lr, seed=4)
    return sc, P, model


@pytest.mark.parametrize("lanes", [1, 16, 33, 100])
def test_learned_decode_parity(ctx, toy, lanes):
    sc, P, model = toy
    buf = S.encode(None, None, mode=S.MODE_LEARNED, depth=10, lanes=lanes, model=model, prep=P)
    st, attr, pos, crd, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK, sgs.lib().sgs_strerror(st)
    assert same_bits(attr, P.attr) and same_bits(pos, P.pos) and np.array_equal(crd, P.coord)


def _random_model(seed):
    rng = np.random.default_rng(seed)
    return dict(w1=rng.integers(-127, 128, (64, 4)), b1=rng.integers(-3000, 3000, (56, 64)),
                w2=rng.integers(-127, 128, (64, 64)), b2=rng.integers(-20000, 20000, 64),
                w3=rng.integers(-127, 128, (256, 64)), b3=rng.integers(-(1 << 23), 1 << 23, 256),
                m1=int(rng.integers(1, 1 << 30)), sh1=int(rng.integers(20, 32)),
                m2=int(rng.integers(1, 1 << 30)), sh2=int(rng.integers(24, 36)),
                ms=int(rng.integers(1, 1 << 24)), ss=int(rng.integers(0, 25)))


def _shaped_model(seed, short12, short3, edge=False):
    """A valid integer model on either side of the decoder's exact shortcuts: short12 keeps
    sh1, sh2 <= 32, m <= 2^sh and |b2| < 2^21 (else one of them is broken), short3 keeps
    |b3| < 2^21 (else one bias sits at 2^21); edge puts the values on the boundaries."""
    rng = np.random.default_rng(100 + seed)
    lim = (1 << 21) - 1
    b2 = rng.integers(-20000, 20000, 64)
    b3 = rng.integers(-(1 << 19), 1 << 19, 256)
    sh1, sh2 = int(rng.integers(20, 31)), int(rng.integers(24, 32))
    m1 = int((127 << sh1) // 30000)
    m2 = int((127 << sh2) // 900000)
    if edge:
        sh2, m1 = 32, 1 << sh1
        m2 = int((127 << sh2) // 900000)
        b2[:2] = (lim, -lim)
        b3[:2] = (lim, -lim)
    if not short12:
        if seed % 3 == 0:
            b2[3] = 1 << 21
        if seed % 3 == 1:
            m1 = (1 << sh1) + 1
        if seed % 3 == 2:
            sh2, m2 = 33, int((127 << 33) // 900000)
    if not short3:
        b3[5] = 1 << 21
    return dict(w1=rng.integers(-127, 128, (64, 4)), b1=rng.integers(-3000, 3000, (56, 64)),
                w2=rng.integers(-127, 128, (64, 64)), b2=b2, w3=rng.integers(-127, 128, (256, 64)), b3=b3,
                m1=m1, sh1=sh1, m2=m2, sh2=sh2, ms=int(rng.integers(200, 4000)), ss=16)


@pytest.mark.parametrize("short12,short3,edge", [(True, True, False), (True, False, False), (False, True, False),
                                                 (False, False, False), (True, True, True)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_learned_decode_both_sides_of_the_shortcuts(ctx, toy, short12, short3, edge, seed):
    """The decoder's exact shortcuts (bias folded into the accumulators, short requantisation)
    and the general forms decode to the oracle's values bit for bit, at the limits too."""
    sc, P, _ = toy
    m = _shaped_model(seed, short12, short3, edge)
    buf = S.encode(None, None, mode=S.MODE_LEARNED, depth=10, lanes=40, model=m, prep=P)
    st, attr, pos, _, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_learned_decode_random_integer_models(ctx, toy, seed):
    """Arbitrary valid integer models: extreme logits, saturated activations, near-certain
    and near-uniform CDFs all decode bit-exactly."""
    sc, P, _ = toy
    m = _random_model(seed)
    buf = S.encode(None, None, mode=S.MODE_LEARNED, depth=10, lanes=40, model=m, prep=P)
    st, attr, pos, _, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos)


def test_learned_encoder_bytes_match_oracle(ctx, toy):
    sc, P, model = toy
    for lanes in (16, 45):
        want = S.encode(sc.pos, sc.attr, mode=S.MODE_LEARNED, depth=10, lanes=lanes, model=model)
        got = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_LEARNED, depth=10, lanes=lanes,
                               model=S.model_bytes(model), ctx=ctx)
        assert got == want


def test_learned_corrupt_model_flagged(ctx, toy):
    sc, P, model = toy
    buf = bytearray(S.encode(None, None, mode=S.MODE_LEARNED, depth=10, lanes=16, model=model, prep=P))
    h = S.parse_header(bytes(buf))
    buf[h["off_attr_tab"] + 4:h["off_attr_tab"] + 8] = (60).to_bytes(4, "little")  # sh1 out of range
    st, _, _, _, _ = gpu_decode(ctx, bytes(buf))
    assert st == sgs.E_CORRUPT


# ----------------------------------------------------------------------------- training

def test_training_gradients_match_fp64(ctx):
    sc = make_scene(5000, 31)
    tokens = sgs.scene_tokens(sc.pos, sc.attr, 11)
    lanes = 24
    lr = S.lane_bounds(tokens.shape[0], lanes)
    w = kaiming_init(9)
    pos = M.sample_positions(13, 0, 4096, tokens.shape[0] * 56)
    u, c, s, _, _ = M.contexts(tokens, lr, pos)
    loss64, g64 = M.forward_backward({k: np.asarray(v, np.float64) for k, v in w.items()}, u, c, s)
    dev = torch.device("cuda", 0)
    grad = torch.zeros(sgs.WEIGHTS_FLOATS, device=dev)
    loss32 = sgs.sgs_train_grad(ctx, torch.from_numpy(tokens).to(dev), tokens.shape[0], lanes,
                                torch.from_numpy(pos).to(dev), torch.from_numpy(sgs.pack_weights(w)).to(dev), grad)
    g32 = sgs.unpack_weights(grad.cpu().numpy())
    assert abs(loss32 - loss64) / loss64 < 1e-5
    for k in M.PARAMS:
        assert_close(g32[k], g64[k], 'gradient ' + k)


def test_training_steps_match_fp64(ctx):
    sc = make_scene(4000, 32)
    tokens = sgs.scene_tokens(sc.pos, sc.attr, 11)
    lanes = 8
    init = kaiming_init(10)
    p64, losses64 = M.train(init, tokens, S.lane_bounds(tokens.shape[0], lanes), 5, 2048, seed=6, lr=1e-3)
    dev = torch.device("cuda", 0)
    w = torch.from_numpy(sgs.pack_weights(init)).to(dev)
    adam = torch.zeros(2 * sgs.WEIGHTS_FLOATS, device=dev)
    losses = torch.zeros(5, device=dev)
    sgs.sgs_train(ctx, torch.from_numpy(tokens).to(dev), tokens.shape[0], lanes, w, adam, steps=5,
                  batch=2048, seed=6, lr=1e-3, loss_dev=losses)
    w32 = sgs.unpack_weights(w.cpu().numpy())
    for k in M.PARAMS:
        assert_close(w32[k], p64[k], 'weights ' + k)
    assert np.allclose(losses.cpu().numpy(), losses64, rtol=1e-4)


def _gain(ctx, rho, n=200_000, steps=400):
    from paper_2607_12656_b300 import learned
    sc = make_scene(n, 77, rho)
    lanes = 1024
    model = learned.train_and_freeze(ctx, sc, 14, lanes, steps=steps, batch=65536, seed=2, lr=3e-3)
    lb = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_LEARNED, depth=14, lanes=lanes, model=model, ctx=ctx)
    sb = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=14, lanes=lanes)
    li, si = sgs.scene_query(lb), sgs.scene_query(sb)
    # attribute payload + its tables or model
    lbytes = li.total_len - li.off[7]
    sbytes = si.total_len - si.off[7]
    return sc, lb, lbytes, sbytes


def test_learned_gain_over_channel_wise(ctx):
    """The trained context model codes the spatially correlated scene in fewer bytes than
    channel-wise static coding (model bytes included), and decodes to identical values; on
    white (rho = 0) attributes it gains nothing beyond its own overhead."""
    sc, lb, lbytes, sbytes = _gain(ctx, 0.8)
    assert lbytes < 0.97 * sbytes, (lbytes, sbytes)
    P = S.prepare(sc.pos, sc.attr, 14, 8)
    st, attr, pos, _, _ = gpu_decode(ctx, lb)
    assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos)
    _, _, l0, s0 = _gain(ctx, 0.0)
    assert l0 > 0.98 * s0, (l0, s0)


def test_full_size_learned_scene(ctx):
    """1M Gaussians, depth 16, 4,096 lanes, model trained 2,000 steps of 65,536 tokens: every
    decoded value equals the oracle's; sampled groups' bytes equal the oracle encoder's and the
    oracle decodes them to the same tokens."""
    from paper_2607_12656_b300 import learned
    sc = make_scene(1_000_000, 2000)
    lanes = 4096
    model = learned.train_and_freeze(ctx, sc, 16, lanes, steps=2000, batch=65536, seed=1)
    buf = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_LEARNED, depth=16, lanes=lanes, model=model, ctx=ctx)
    P = S.prepare(sc.pos, sc.attr, 16, 8)
    st, attr, pos, _, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos)
    h = S.parse_header(buf)
    m = S.parse_model(buf, h["off_attr_tab"])
    G = (lanes + 31) // 32
    goff = np.frombuffer(buf, "<u8", G + 1, h["off_attr_grp"])
    gw = np.frombuffer(buf, "<u4", G, h["off_attr_grp"] + 8 * (G + 1))
    pay = buf[h["off_attr_pay"]:]
    lr = S.lane_bounds(P.n_rows, lanes)
    q = P.q.astype(np.uint8)
    for g in (0, 57, G - 1):
        lo, hi = 32 * g, min(lanes, 32 * g + 32)
        f, c = S.learned_fc(m, q, lr, lo, hi)
        ls = (lr[lo:hi + 1] - lr[lo]) * 56
        want, _, _ = S.rans_encode(ls, f, c)
        assert pay[int(goff[g]):int(goff[g + 1])] == want
        dec = S.rans_decode_learned(m, lr, lo, hi, pay, goff, gw, P.n_rows)
        assert np.array_equal(dec[lr[lo]:lr[hi]], q[lr[lo]:lr[hi]])


def test_training_resumes_exactly(ctx):
    """Checkpoint and resume: 3 steps, then 3 more from the saved weights and Adam moments at
    step0 = 3, give the same weights, bit for bit, as 6 uninterrupted steps (the sampler and
    the bias corrections are indexed by the global step), and both agree element-wise with
    the fp64 oracle's 6 steps."""
    sc = make_scene(4000, 33)
    tokens = sgs.scene_tokens(sc.pos, sc.attr, 11)
    lanes = 8
    init = kaiming_init(11)
    dev = torch.device("cuda", 0)
    tok = torch.from_numpy(tokens).to(dev)
    whole = torch.from_numpy(sgs.pack_weights(init)).to(dev)
    adam = torch.zeros(2 * sgs.WEIGHTS_FLOATS, device=dev)
    sgs.sgs_train(ctx, tok, tokens.shape[0], lanes, whole, adam, steps=6, batch=2048, seed=7, lr=1e-3)
    part = torch.from_numpy(sgs.pack_weights(init)).to(dev)
    adam2 = torch.zeros(2 * sgs.WEIGHTS_FLOATS, device=dev)
    sgs.sgs_train(ctx, tok, tokens.shape[0], lanes, part, adam2, steps=3, batch=2048, seed=7, lr=1e-3)
    saved_w, saved_adam = part.cpu().clone(), adam2.cpu().clone()  # the checkpoint
    part, adam2 = saved_w.to(dev), saved_adam.to(dev)
    sgs.sgs_train(ctx, tok, tokens.shape[0], lanes, part, adam2, steps=3, batch=2048, seed=7, lr=1e-3, step0=3)
    assert torch.equal(part.view(torch.int32), whole.view(torch.int32))
    assert torch.equal(adam2.view(torch.int32), adam.view(torch.int32))
    p64, _ = M.train(init, tokens, S.lane_bounds(tokens.shape[0], lanes), 6, 2048, seed=7, lr=1e-3)
    w32 = sgs.unpack_weights(part.cpu().numpy())
    for k in M.PARAMS:
        assert_close(w32[k], p64[k], 'resumed weights ' + k)


def test_bounded_wait_times_out_and_context_recovers(ctx, toy):
    """Failure detection without a GPU fault: with a poll budget of 1 the decoder's first wait
    that is not already satisfied gives up, the decode reports SGS_E_TIMEOUT through
    sgs_sync, every warp leaves, and the same context then decodes the scene bit-exactly
    with the default budget."""
    sc, P, model = toy
    buf = S.encode(None, None, mode=S.MODE_LEARNED, depth=10, lanes=64, model=model, prep=P)
    ctx.set_wait_limit(1)
    try:
        st, _, _, _, _ = gpu_decode(ctx, buf)
    finally:
        ctx.set_wait_limit(0)
    assert st == sgs.E_TIMEOUT, sgs.lib().sgs_strerror(st)
    st, attr, pos, crd, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos) and np.array_equal(crd, P.coord)
