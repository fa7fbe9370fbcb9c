"""Learned constitutive surrogate: device kernels against the FP64 reference network, training on
return-map data generated by the solver, and the fused inference with exact fallback."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_2602_15149_b300 import surrogate, tlsph, workloads as W

pytestmark = pytest.mark.gpu


def identity_norm():
    n = np.zeros(96, np.float32)
    n[16:32] = 1.0
    n[48:64] = 1.0
    n[64:80] = -np.inf
    n[80:96] = np.inf
    return n


def bf16_round(a):
    """Round float arrays to the nearest bfloat16 (what the tensor cores see)."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.mark.parametrize("path", [tlsph.TENSOR_TCGEN05, tlsph.TENSOR_MMA_SYNC])
def test_forward_matches_reference(torch, path):
    params = ref.init_params(seed=3)
    params = [(bf16_round(W).astype(np.float64), b) for W, b in params]
    net = tlsph.MLP(batch=256)
    net.set_tensor_path(path)
    net.set_params(tlsph.pack_params(params))
    net.set_normalization(identity_norm())
    x = np.random.default_rng(0).normal(size=(300, 16)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    net.forward(xd, yd)
    out_ref, _ = ref.forward(params, bf16_round(x).astype(np.float64))
    err = np.linalg.norm(yd.cpu().numpy() - out_ref) / np.linalg.norm(out_ref)
    assert err < 1e-2, err


def test_tensor_paths_agree(torch):
    """tcgen05 (TMEM accumulators) and mma.sync give the same network output up to summation
    order, on a ragged row count that spans many tiles."""
    params = ref.init_params(seed=9)
    net = tlsph.MLP(batch=256)
    net.set_params(tlsph.pack_params(params))
    net.set_normalization(identity_norm())
    x = torch.from_numpy(np.random.default_rng(4).normal(size=(100_003, 16)).astype(np.float32)).cuda()
    outs = []
    for path in (tlsph.TENSOR_TCGEN05, tlsph.TENSOR_MMA_SYNC):
        net.set_tensor_path(path)
        y = torch.empty_like(x)
        net.forward(x, y)
        outs.append(y.cpu().numpy())
    err = np.linalg.norm(outs[0] - outs[1]) / np.linalg.norm(outs[1])
    print("tcgen05 vs mma.sync: rel-L2", err, "bit-identical", np.array_equal(outs[0], outs[1]))
    assert np.all(np.isfinite(outs[0])) and err < 2e-3, err


def test_gradients_match_reference(torch):
    params = ref.init_params(seed=5)
    params = [(bf16_round(W).astype(np.float64), b) for W, b in params]
    net = tlsph.MLP(batch=512)
    net.set_params(tlsph.pack_params(params))
    net.set_normalization(identity_norm())
    rng = np.random.default_rng(1)
    x = bf16_round(rng.normal(size=(512, 16)))
    y = rng.normal(size=(512, 16)).astype(np.float32)
    loss, g = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    loss_ref, grads_ref = ref.loss_and_grads(params, x.astype(np.float64), y.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref
    for (gW, gb), (rW, rb) in zip(tlsph.unpack_params(g), grads_ref):
        for a, b in ((gW, rW), (gb, rb)):
            cos = float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b)))
            rel = float(np.linalg.norm(a - b) / np.linalg.norm(b))
            assert cos > 0.999 and rel < 5e-2, (cos, rel)


@pytest.mark.parametrize("batch", [2048, 512, 272])
def test_training_gemm_paths_agree(torch, batch):
    """The training GEMMs on tcgen05 (TMEM accumulators, one CTA per 128 x 128 tile; a batch of 272 rows
    leaves a ragged last tile) and on mma.sync give the same loss and gradients up to summation order,
    and a few Adam steps on either path move the parameters alike."""
    params = ref.init_params(seed=7)
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.normal(size=(batch, 16)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.normal(size=(batch, 16)).astype(np.float32)).cuda()
    out = {}
    for path in (tlsph.TENSOR_TCGEN05, tlsph.TENSOR_MMA_SYNC):
        net = tlsph.MLP(batch=batch)
        net.set_tensor_path(path)
        net.set_params(tlsph.pack_params(params))
        net.set_normalization(identity_norm())
        loss, g = net.gradients(x, y)
        for _ in range(5):
            net.train_step(x, y, lr=1e-3)
        out[path] = (loss, g, net.get_params())
    (l0, g0, p0), (l1, g1, p1) = out[tlsph.TENSOR_TCGEN05], out[tlsph.TENSOR_MMA_SYNC]
    assert abs(l0 - l1) <= 1e-3 * abs(l1)
    assert np.linalg.norm(g0 - g1) <= 1e-2 * np.linalg.norm(g1)
    assert np.linalg.norm(p0 - p1) <= 1e-3 * np.linalg.norm(p1)


@pytest.fixture(scope="module")
def trained(torch):
    """A network trained on return-map samples of a small J2 block (same recipe as the 1M block)."""
    case = W.block_3d(nx=24, ny=24, nz=12)
    x, y, pn = surrogate.generate_samples(case, n_target=400_000, steps=1200, every=10, stride_elastic=2)
    n = x.shape[0]
    ntr = int(0.9 * n)
    net, info = surrogate.train(x[:ntr], y[:ntr], epochs=60, batch=1024, lr=2e-3)
    return case, net, info, (x[ntr:], y[ntr:], pn[ntr:]), (x[:ntr], y[:ntr])


def test_samples_are_deterministic(torch):
    case = W.block_3d(nx=14, ny=12, nz=9)
    a = surrogate.generate_samples(case, n_target=20_000, steps=300, every=30, stride_elastic=1)
    b = surrogate.generate_samples(case, n_target=20_000, steps=300, every=30, stride_elastic=1)
    assert a[0].shape[0] > 1000
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    # elastic rows carry exactly zero corrections (stress and state); plastic rows a positive
    # eps_p increment
    y = a[1].cpu().numpy()
    assert np.all(y[:, 15] >= 0.0)
    zero = np.all(y == 0.0, axis=1)
    assert zero.any() and (y[:, 15] > 0.0).any()
    assert np.all(a[2].cpu().numpy() > 0.0)


def test_training_learns_the_return_map(trained):
    case, net, info, (xv, yv, pv), _ = trained
    assert info["samples"] > 50_000
    err = surrogate.stress_error(net, xv, yv, pv, case.materials[0].sigma_y0)
    print("held-out stress error", err, info)
    assert err["inside_fraction"] > 0.95
    assert err["mean"] <= 1e-2


def test_fallback_outside_envelope_is_the_exact_step(torch):
    case = W.block_3d(nx=14, ny=12, nz=9)
    exact = tlsph.from_case(case)
    exact.step(120)
    net = tlsph.MLP(batch=256)
    norm = identity_norm()
    norm[64:80], norm[80:96] = np.inf, -np.inf  # empty envelope: every particle falls back
    net.set_normalization(norm)
    g = tlsph.from_case(case)
    g.set_surrogate(net)
    g.step(120)
    assert np.array_equal(g.read_state("U"), exact.read_state("U"))
    used, fallback, elastic = g.surrogate_counts()
    assert used == 0 and fallback == 120 * case.n and elastic == 0


@pytest.mark.parametrize("path", [tlsph.TENSOR_TCGEN05, tlsph.TENSOR_MMA_SYNC])
def test_indefinite_network_state_is_refused(torch, path):
    """A network whose b_e correction is -10 I would leave C_p^-1 indefinite: every output is refused,
    nothing of it is written, and the exact return map serves the particle, so the run is the exact
    one bit for bit and all updates count as served exactly."""
    case = W.block_3d(nx=14, ny=12, nz=9)
    exact = tlsph.from_case(case)
    exact.step(60)
    net = tlsph.MLP(batch=256)
    net.set_params(tlsph.pack_params(ref.init_params(seed=2)))
    net.set_tensor_path(path)
    norm = identity_norm()  # out = out_mean + out_std * network
    norm[48 + 9:48 + 12] = 1e-30  # (a std must be positive)
    norm[32 + 9:32 + 12] = -10.0  # db = -10 I whatever the network says
    net.set_normalization(norm)
    g = tlsph.from_case(case)
    g.set_surrogate(net)
    g.step(60)
    assert np.array_equal(g.read_state("U"), exact.read_state("U"))
    assert np.array_equal(g.read_state("EPSP"), exact.read_state("EPSP"))
    used, fallback, elastic = g.surrogate_counts()
    assert used == 0 and fallback == 60 * case.n and elastic == 0


@pytest.mark.parametrize("scope,path", [(tlsph.SURROGATE_ALL, tlsph.TENSOR_TCGEN05),
                                        (tlsph.SURROGATE_PLASTIC, tlsph.TENSOR_TCGEN05),
                                        (tlsph.SURROGATE_ALL, tlsph.TENSOR_MMA_SYNC)])
def test_surrogate_step_tracks_exact_step(trained, scope, path):
    """400 steps with the network in the J2 update stay within 1% (rel-L2 of u) of the exact run.
    The held-out stress error is ~0.5%; the state enters as increments, so the error does not
    random-walk in the state."""
    case, net, _, _, _ = trained
    exact = tlsph.from_case(case)
    sur = tlsph.from_case(case)
    net.set_tensor_path(path)
    sur.set_surrogate(net, scope)
    net.set_tensor_path(tlsph.TENSOR_TCGEN05)
    exact.step(400)
    sur.step(400)
    used, outside, elastic = sur.surrogate_counts()
    ue, us = exact.read_state("U"), sur.read_state("U")
    err = float(np.linalg.norm(us - ue) / np.linalg.norm(ue))
    ep_e, ep_s = exact.read_state("EPSP"), sur.read_state("EPSP")
    print("scope", scope, "path", path, "surrogate vs exact: rel-L2(u)", err, "max |d eps_p|", np.abs(ep_s - ep_e).max(),
          "rows by network", used, "outside", outside, "elastic", elastic)
    assert used + outside + elastic == 400 * case.n
    if scope == tlsph.SURROGATE_ALL:
        assert elastic == 0 and used > 0.9 * 400 * case.n
    else:
        assert used > 0 and elastic > 0
    assert err < 1e-2


def test_network_file_round_trip_and_load_surrogate(trained, tmp_path):
    """A trained network written to a file and read back gives bit-identical outputs, and a context that
    loads the file steps bit-identically to one given the network object; a foreign file is refused."""
    import torch as t
    case, net, _, _, _ = trained
    path = tmp_path / "net.tlsphmlp"
    net.save(str(path))
    other = tlsph.MLP(batch=256)
    other.load(str(path))
    x = t.from_numpy(np.random.default_rng(3).normal(size=(300, 16)).astype(np.float32)).cuda()
    y1, y2 = t.empty((300, 16), device="cuda"), t.empty((300, 16), device="cuda")
    net.forward(x, y1)
    other.forward(x, y2)
    assert t.equal(y1, y2)
    a, b = tlsph.from_case(case), tlsph.from_case(case)
    a.set_surrogate(net, tlsph.SURROGATE_ALL)
    b.load_surrogate(str(path), tlsph.SURROGATE_ALL)
    a.step(50)
    b.step(50)
    assert np.array_equal(a.read_state("U"), b.read_state("U"))
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a network")
    with pytest.raises(tlsph.TLSPHError):
        b.load_surrogate(str(bad))
    with pytest.raises(tlsph.TLSPHError):
        other.load(str(tmp_path / "missing.bin"))
