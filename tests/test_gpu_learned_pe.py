"""GPU parity of the position-aware learned mode (Fourier positional embedding + Laplace head):
decode bit-exact against the oracle (oracle-trained and arbitrary integer models, every
output variant, alone, batched and allocation-free) and the library encoder's bytes against
the oracle's."""
import numpy as np
import pytest

from oracle import model as M
from oracle import model_pe as E
from oracle import scene as S
from paper_2607_12656_b300 import sgs
from paper_2607_12656_b300.scenegen import kaiming_init_pe, make_scene

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
    p, _ = E.train(kaiming_init_pe(2), q, lr, P.coord, 10, 60, 2048, seed=4, lr=3e-3)
    model = E.freeze({k: v.astype(np.float32) for k, v in p.items()}, q, lr, P.coord, 10, seed=4)
    return sc, P, model


def _decode(ctx, buf, coords=True, out_index=None):
    info = sgs.scene_query(buf)
    ctx.reserve(info.scratch_bytes)
    bits = torch.frombuffer(bytearray(buf), dtype=torch.uint8).cuda()
    n = info.n_rows
    attr = torch.full((56, max(n, 1)), float("nan"), device="cuda")
    pos = torch.full((3, max(n, 1)), float("nan"), device="cuda")
    crd = torch.full((3, max(n, 1)), -1, dtype=torch.int32, device="cuda") if coords else None
    oi = None if out_index is None else torch.from_numpy(out_index.astype(np.int32)).cuda()
    sgs.scene_decode(ctx, bits, info, attr, pos, crd, oi)
    st = ctx.sync()
    return st, attr.cpu().numpy()[:, :n], pos.cpu().numpy()[:, :n]


@pytest.mark.parametrize("lanes", [1, 16, 33, 100, 300])
def test_decode_parity(ctx, toy, lanes):
    sc, P, model = toy
    buf = S.encode(None, None, mode=S.MODE_LEARNED_PE, depth=10, lanes=lanes, model=model, prep=P)
    st, attr, pos, crd, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK, sgs.lib().sgs_strerror(st)
    assert same_bits(attr, P.attr) and same_bits(pos, P.pos) and np.array_equal(crd, P.coord)


def test_decode_without_coordinates_and_permuted(ctx, toy):
    """The model reads the voxels from scratch when the caller asks for no coordinates, and
    at the permuted columns when an out_index is given."""
    sc, P, model = toy
    buf = S.encode(None, None, mode=S.MODE_LEARNED_PE, depth=10, lanes=40, model=model, prep=P)
    st, attr, pos = _decode(ctx, buf, coords=False)
    assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos)
    perm = np.random.default_rng(3).permutation(P.n_rows)
    for coords in (True, False):
        st, attr, pos = _decode(ctx, buf, coords=coords, out_index=perm)
        assert st == sgs.OK and same_bits(attr[:, perm], P.attr) and same_bits(pos[:, perm], P.pos)


def _random_model(seed):
    rng = np.random.default_rng(seed)
    return dict(w1=rng.integers(-127, 128, (64, 80)), b1=rng.integers(-(1 << 22), 1 << 22, (56, 64)),
                s1=np.float32(rng.uniform(1e-6, 1e-3)), w2=rng.integers(-127, 128, (64, 64)),
                b2=rng.integers(-(1 << 20), 1 << 20, 64), s2=np.float32(rng.uniform(1e-5, 1e-3)),
                w3=rng.integers(-127, 128, (2, 64)), b3=rng.integers(-(1 << 20), 1 << 20, 2),
                smu=np.float32(rng.uniform(1e-4, 0.1)), slr=np.float32(rng.uniform(1e-5, 0.01)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_decode_random_integer_models(ctx, toy, seed):
    """Saturated activations, means at the range ends, the narrowest and widest rates."""
    sc, P, _ = toy
    buf = S.encode(None, None, mode=S.MODE_LEARNED_PE, depth=10, lanes=37, model=_random_model(seed), prep=P)
    st, attr, pos, _, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos)


def test_encoder_bytes_match_oracle(ctx, toy):
    sc, P, model = toy
    for lanes in (16, 45):
        want = S.encode(sc.pos, sc.attr, mode=S.MODE_LEARNED_PE, depth=10, lanes=lanes, model=model)
        got = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_LEARNED_PE, depth=10, lanes=lanes,
                               model=E.model_bytes(model), ctx=ctx)
        assert got == want


def test_corrupt_model_and_payload_flagged(ctx, toy):
    sc, P, model = toy
    buf = bytearray(S.encode(None, None, mode=S.MODE_LEARNED_PE, depth=10, lanes=16, model=model, prep=P))
    h = S.parse_header(bytes(buf))
    bad = bytearray(buf)
    bad[h["off_attr_tab"]:h["off_attr_tab"] + 4] = np.float32(np.nan).tobytes()  # s1 = NaN
    assert gpu_decode(ctx, bytes(bad))[0] == sgs.E_CORRUPT
    bad = bytearray(buf)
    bad[h["off_attr_tab"] + 32:h["off_attr_tab"] + 36] = (1 << 23).to_bytes(4, "little")  # B1 too large
    assert gpu_decode(ctx, bytes(bad))[0] == sgs.E_CORRUPT
    bad = bytearray(buf)
    for k in range(h["off_attr_pay"], min(h["off_attr_pay"] + 64, h["total"])):
        bad[k] ^= 0x5A
    assert gpu_decode(ctx, bytes(bad))[0] == sgs.E_CORRUPT
    # the library refuses to encode with an invalid model
    m = bytearray(E.model_bytes(model))
    m[0:4] = np.float32(-1.0).tobytes()
    with pytest.raises(sgs.SgsError):
        sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_LEARNED_PE, depth=10, lanes=16, model=bytes(m), ctx=ctx)


def test_deep_scene_parity(ctx):
    """Depth 18 with duplicates: every band of the embedding sees fine phases."""
    sc = make_scene(20000, 44)
    P = S.prepare(sc.pos, sc.attr, 18, 8)
    m = _random_model(7)
    buf = S.encode(None, None, mode=S.MODE_LEARNED_PE, depth=18, lanes=200, model=m, prep=P)
    st, attr, pos, crd, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK and same_bits(attr, P.attr) and np.array_equal(crd, P.coord)


def test_batched_and_noalloc_parity(ctx, toy):
    """Position-aware scenes in a batch beside a static one (the model's stage follows the
    octree walk), and through the allocation-free entry point."""
    sc, P, model = toy
    bufs = [S.encode(None, None, mode=S.MODE_LEARNED_PE, depth=10, lanes=40, model=model, prep=P),
            S.encode(None, None, mode=S.MODE_STATIC, depth=10, lanes=64, prep=P),
            S.encode(None, None, mode=S.MODE_LEARNED_PE, depth=10, lanes=7, model=_random_model(3), prep=P)]
    items = []
    for j, b in enumerate(bufs):
        info = sgs.scene_query(b)
        bits = torch.frombuffer(bytearray(b), dtype=torch.uint8).cuda()
        attr = torch.full((56, info.n_rows), float("nan"), device="cuda")
        pos = torch.full((3, info.n_rows), float("nan"), device="cuda")
        items.append((bits, info, attr, pos))
    c = sgs.Context(0, 0)
    plan = sgs.BatchPlan(c, items)
    plan.run()
    assert c.sync() == sgs.OK and plan.status() == [sgs.OK] * 3
    for it in items:
        assert same_bits(it[2].cpu().numpy(), P.attr) and same_bits(it[3].cpu().numpy(), P.pos)
    plan.close()
    c.close()
    info = sgs.scene_query(bufs[0])
    bits = torch.frombuffer(bytearray(bufs[0]), dtype=torch.uint8).cuda()
    attr = torch.full((56, info.n_rows), float("nan"), device="cuda")
    pos = torch.full((3, info.n_rows), float("nan"), device="cuda")
    assert sgs.scene_decode_noalloc(bits, info, attr, pos) == sgs.OK
    assert same_bits(attr.cpu().numpy(), P.attr)


# ----------------------------------------------------------------------------- training

def test_training_gradients_match_fp64(ctx):
    sc = make_scene(5000, 31)
    tokens, coord = sgs.scene_rows(sc.pos, sc.attr, 11)
    lanes = 24
    lr = S.lane_bounds(tokens.shape[0], lanes)
    w = kaiming_init_pe(9)
    w["w3"] = w["w3"] * 10.0  # spread the heads: every branch of the Laplace gradient is used
    pos = M.sample_positions(13, 0, 4096, tokens.shape[0] * 56)
    u, c, phi, s = E.batch(tokens, lr, E.phi_q(coord, 11), pos)
    loss64, g64 = E.forward_backward({k: np.asarray(v, np.float64) for k, v in w.items()}, u, c, phi, s)
    dev = torch.device("cuda", 0)
    grad = torch.zeros(sgs.WEIGHTS_PE_FLOATS, device=dev)
    loss32 = sgs.sgs_train_pe_grad(ctx, torch.from_numpy(tokens).to(dev), torch.from_numpy(coord.view(np.int32)).to(dev),
                                   11, tokens.shape[0], lanes, torch.from_numpy(pos).to(dev),
                                   torch.from_numpy(sgs.pack_weights_pe(w)).to(dev), grad)
    g32 = sgs.unpack_weights_pe(grad.cpu().numpy())
    assert abs(loss32 - loss64) / loss64 < 1e-5
    for k in E.PARAMS:
        assert_close(g32[k], g64[k], 'gradient ' + k)


def test_training_steps_match_fp64(ctx):
    sc = make_scene(4000, 32)
    tokens, coord = sgs.scene_rows(sc.pos, sc.attr, 11)
    lanes = 8
    init = kaiming_init_pe(10)
    p64, losses64 = E.train(init, tokens, S.lane_bounds(tokens.shape[0], lanes), coord, 11, 5, 2048, seed=6, lr=1e-3)
    dev = torch.device("cuda", 0)
    w = torch.from_numpy(sgs.pack_weights_pe(init)).to(dev)
    adam = torch.zeros(2 * sgs.WEIGHTS_PE_FLOATS, device=dev)
    losses = torch.zeros(5, device=dev)
    sgs.sgs_train_pe(ctx, torch.from_numpy(tokens).to(dev), torch.from_numpy(coord.view(np.int32)).to(dev), 11,
                     tokens.shape[0], lanes, w, adam, steps=5, batch=2048, seed=6, lr=1e-3, loss_dev=losses)
    w32 = sgs.unpack_weights_pe(w.cpu().numpy())
    for k in E.PARAMS:
        assert_close(w32[k], p64[k], 'weights ' + k)
    assert np.allclose(losses.cpu().numpy(), losses64, rtol=1e-4)


def test_trained_model_codes_better_than_channel_wise(ctx):
    """End to end on the device: train, freeze, encode, decode; the position-aware model's
    attribute bytes undercut static channel-wise coding on a spatially correlated scene, and
    the decode matches the oracle."""
    from paper_2607_12656_b300 import learned
    sc = make_scene(100_000, 77)
    lanes = 1024
    model = learned.train_and_freeze_pe(ctx, sc, 14, lanes, steps=300, batch=65536, seed=2, lr=3e-3)
    pb = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_LEARNED_PE, depth=14, lanes=lanes, model=model, ctx=ctx)
    sb = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_STATIC, depth=14, lanes=lanes)
    pi, si = sgs.scene_query(pb), sgs.scene_query(sb)
    assert pi.total_len - pi.off[7] < 0.97 * (si.total_len - si.off[7])
    P = S.prepare(sc.pos, sc.attr, 14, 8)
    st, attr, pos, crd, _ = gpu_decode(ctx, pb)
    assert st == sgs.OK and same_bits(attr, P.attr) and np.array_equal(crd, P.coord)


def test_full_size_scene(ctx):
    """The bench's configuration: 1M Gaussians, depth 16, 28,125 lanes (W = 32), model trained
    2,000 steps of 65,536 tokens on the device; every decoded value equals the oracle's;
    sampled groups' bytes equal the oracle encoder's and the oracle decodes them to the same
    tokens."""
    from paper_2607_12656_b300 import learned
    sc = make_scene(1_000_000, 2000)
    lanes = 28125
    model = learned.train_and_freeze_pe(ctx, sc, 16, lanes, steps=2000, batch=65536, seed=1)
    buf = sgs.scene_encode(sc.pos, sc.attr, mode=sgs.MODE_LEARNED_PE, depth=16, lanes=lanes, model=model, ctx=ctx)
    P = S.prepare(sc.pos, sc.attr, 16, 8)
    st, attr, pos, crd, _ = gpu_decode(ctx, buf)
    assert st == sgs.OK and same_bits(attr, P.attr) and same_bits(pos, P.pos) and np.array_equal(crd, P.coord)
    h = S.parse_header(buf)
    m = E.parse_model(buf, h["off_attr_tab"])
    G = (lanes + 31) // 32
    goff = np.frombuffer(buf, "<u8", G + 1, h["off_attr_grp"])
    gw = np.frombuffer(buf, "<u4", G, h["off_attr_grp"] + 8 * (G + 1))
    pay = buf[h["off_attr_pay"]:]
    lr = S.lane_bounds(P.n_rows, lanes)
    q = P.q.astype(np.uint8)
    for g in (0, 411, G - 1):
        lo, hi = 32 * g, min(lanes, 32 * g + 32)
        f, c = E.token_fc(m, q, lr, P.coord, 16, int(lr[lo]), int(lr[hi]))
        want, _, _ = S.rans_encode((lr[lo:hi + 1] - lr[lo]) * 56, f, c)
        assert pay[int(goff[g]):int(goff[g + 1])] == want
        dec = S.rans_decode_pe(m, P.coord, 16, lr, pay, goff, gw, lo, hi)
        assert np.array_equal(dec[lr[lo]:lr[hi]], q[lr[lo]:lr[hi]])


def test_training_resumes_exactly(ctx):
    """Checkpoint and resume of the position-aware model: 3 + 3 steps (step0 = 3 from the
    saved weights and moments) equal 6 uninterrupted steps bit for bit, and the fp64
    oracle's 6 steps element-wise."""
    sc = make_scene(4000, 34)
    tokens, coord = sgs.scene_rows(sc.pos, sc.attr, 11)
    lanes = 8
    init = kaiming_init_pe(12)
    dev = torch.device("cuda", 0)
    tok = torch.from_numpy(tokens).to(dev)
    crd = torch.from_numpy(coord.view(np.int32)).to(dev)
    args = (ctx, tok, crd, 11, tokens.shape[0], lanes)
    whole = torch.from_numpy(sgs.pack_weights_pe(init)).to(dev)
    adam = torch.zeros(2 * sgs.WEIGHTS_PE_FLOATS, device=dev)
    sgs.sgs_train_pe(*args, whole, adam, steps=6, batch=2048, seed=8, lr=1e-3)
    part = torch.from_numpy(sgs.pack_weights_pe(init)).to(dev)
    adam2 = torch.zeros(2 * sgs.WEIGHTS_PE_FLOATS, device=dev)
    sgs.sgs_train_pe(*args, part, adam2, steps=3, batch=2048, seed=8, lr=1e-3)
    part, adam2 = part.cpu().clone().to(dev), adam2.cpu().clone().to(dev)
    sgs.sgs_train_pe(*args, part, adam2, steps=3, batch=2048, seed=8, lr=1e-3, step0=3)
    assert torch.equal(part.view(torch.int32), whole.view(torch.int32))
    assert torch.equal(adam2.view(torch.int32), adam.view(torch.int32))
    p64, _ = E.train(init, tokens, S.lane_bounds(tokens.shape[0], lanes), coord, 11, 6, 2048, seed=8, lr=1e-3)
    w32 = sgs.unpack_weights_pe(part.cpu().numpy())
    for k in E.PARAMS:
        assert_close(w32[k], p64[k], 'resumed weights ' + k)
