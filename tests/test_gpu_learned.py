"""GPU tests of the learned penumbra surrogate (this library's addition).

The surrogate's features must equal the oracle's bit for bit; its
tensor-core forward and backward must match the BF16-emulating float64
reference within bounds derived from the arithmetic; training on the GPU
must lower the loss; and with the surrogate switched on the exact parts of
the method (shadow tests, discontinuity codes, off-edge answers, the hard
shadow of silhouette recovery) must not change by one bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import mlp as omlp  # noqa: E402
from oracle import rbsm as orc  # noqa: E402
from tests.test_gpu_parity import dev  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_07793_gb300 import api, surrogate
    return api, surrogate


@pytest.fixture(scope="module")
def scene():
    import rbsm_scenes as sc
    return sc.config2(3, screen=(960, 540))


def _oracle_samples(f):
    ref = orc.evaluate(f.depth, f.x, f.y, f.z, orc.MODE_FILTER)
    edge = ((ref["codes"] >> 9) & 1) == 1
    feat = orc.features(f.depth, f.x[edge], f.y[edge], f.z[edge])
    return feat, ref["vis"][edge]


def test_dataset_matches_oracle_features_and_labels(lib, scene):
    api, S = lib
    f = scene
    samples, count = S.Surrogate.dataset([(dev(f.depth), dev(f.x), dev(f.y), dev(f.z))], capacity=1 << 20)
    got = S.Surrogate.unpack(samples, count)
    feat, labels = _oracle_samples(f)
    assert count == labels.size > 1000
    key = lambda d, lab: np.lexsort((lab, d["gap"], d["fy"], d["fx"], d["bits"]))
    ga, oa = key(got, got["label"]), key(feat, labels)
    for k in ("bits", "fx", "fy", "gap"):
        assert np.array_equal(got[k][ga], feat[k][oa]), k
    assert np.max(np.abs(got["label"][ga].astype(np.float64) - labels[oa])) <= 1e-5


def _bound_forward(P, X):
    """Deviation allowed between the GPU forward and the BF16-emulating
    float64 reference: FP32 accumulation differs from float64 by a few
    ulps of each sum, and when a sum lands within that distance of a BF16
    rounding boundary the two sides round a hidden unit to neighbouring
    BF16 values (at most 2^-7 relative).  The bound allows one such flip in
    h1, carried through W2 and W3, plus a flip of every unit of h2, on top of
    a 1e-4 floor for the accumulation differences."""
    y, c = omlp.forward(P, X, bf16=True)
    w2 = np.abs(c["W2"]).max(axis=1)                     # per h1 unit
    w3 = np.abs(c["W3"]).max(axis=1)                     # per h2 unit
    path1 = (np.abs(c["h1"]) * w2[None, :]).max(axis=1) * np.abs(c["W3"]).sum(axis=0).max()
    path2 = (np.abs(c["h2"]) * w3[None, :]).sum(axis=1)
    return y, 1e-4 + 2.0 ** -7 * (path1 + path2)


def test_forward_matches_reference(lib, scene):
    api, S = lib
    import rbsm_scenes as sc
    feat, labels = _oracle_samples(scene)
    P32 = sc.mlp_init(1)
    net = S.Surrogate(P32)
    samples, n = S.Surrogate.pack(feat, labels)
    out = net.forward(samples, n).cpu().numpy().astype(np.float64)
    P = {k: v.astype(np.float64) for k, v in P32.items()}
    y, bound = _bound_forward(P, omlp.encode(feat))
    diff = np.abs(out - y).max(axis=1)
    assert np.all(diff <= bound), (diff.max(), bound[np.argmax(diff - bound)])
    assert np.mean(diff <= 1e-4) > 0.999


def test_gradient_and_adam_match_reference(lib, scene):
    api, S = lib
    import rbsm_scenes as sc
    feat, labels = _oracle_samples(scene)
    B = 4096
    feat = {k: v[:B] for k, v in feat.items()}
    labels = labels[:B]
    P32 = sc.mlp_init(2)
    net = S.Surrogate(P32)
    samples, n = S.Surrogate.pack(feat, labels)
    order = torch.arange(n, dtype=torch.int32, device="cuda")
    net.grad(samples, order)
    g = S.Surrogate.unflatten(net.read_grad())
    loss_gpu = net.take_loss() / n
    P = {k: v.astype(np.float64) for k, v in P32.items()}
    loss, G = omlp.loss_and_grads(P, omlp.encode(feat), labels, bf16=True)
    assert abs(loss_gpu - loss) <= 1e-3 * loss + 1e-6
    for k in G:
        rel = np.linalg.norm(g[k] - G[k]) / max(np.linalg.norm(G[k]), 1e-12)
        assert rel <= 2e-2, (k, rel)
    # one Adam step on both sides from their own gradients
    net.adam(1e-3)
    after = S.Surrogate.unflatten(net.params())
    M = {k: np.zeros_like(v) for k, v in P.items()}
    V = {k: np.zeros_like(v) for k, v in P.items()}
    omlp.adam_step(P, G, M, V, 1, 1e-3)
    for k in P:
        d = np.abs(after[k] - P[k])
        assert d.max() <= 2e-3 + 1e-6                        # a sign flip of a tiny gradient moves by 2 lr
        assert np.mean(d <= 1e-5) > 0.95


def test_training_lowers_the_loss_and_the_guard_trades_error_for_fallbacks(lib):
    """Train on edge fragments of two scenes, then run the learned batch on a
    third: the exact parts are unchanged bit for bit, accepted answers are
    close to the exact ones on average, and a tighter guard sends more
    fragments to the exact walk."""
    api, S = lib
    import rbsm_scenes as sc
    train = [sc.config2(s, screen=(1280, 720)) for s in (10, 11)]
    data = [(dev(f.depth), dev(f.x), dev(f.y), dev(f.z)) for f in train]
    samples, count = S.Surrogate.dataset(data, capacity=1 << 20)
    net = S.Surrogate(sc.mlp_init(0))
    hist = net.train(samples, count, epochs=4, batch=4096, lr=3e-3)
    assert hist[-1] < 0.6 * hist[0]
    test = sc.config2(12, screen=(1280, 720))
    depth, x, y, z = dev(test.depth), dev(test.x), dev(test.y), dev(test.z)

    def run(surrogate, tau, mode):
        job = api.Job(0, x, y, z, mode=mode, codes=True)
        b = api.Batch([depth], [job], surrogate=surrogate, guard_tau=tau)
        api.rbsm_batch_run(b)
        torch.cuda.synchronize()
        return job, api.rbsm_batch_surrogate_counts(b)

    exact, _ = run(None, 0.0, 2)
    ex_f = exact.vis_filter.cpu().numpy()
    ex_c = exact.codes.cpu().numpy().view(np.uint16)
    edge = ((ex_c >> 9) & 1) == 1
    fallbacks = []
    for tau in (1.0, 0.1, 0.02):
        job, (acc, fb) = run(net, tau, 2)
        f = job.vis_filter.cpu().numpy()
        c = job.codes.cpu().numpy().view(np.uint16)
        assert acc + fb == edge.sum()
        assert np.array_equal(c & 0x1F, ex_c & 0x1F)                   # tests and directions exact
        assert np.array_equal(f[~edge], ex_f[~edge])                   # off-edge answers exact
        learned = ((c >> 10) & 1) == 1
        assert learned.sum() == acc
        assert np.array_equal(f[edge & ~learned], ex_f[edge & ~learned])   # fallbacks are exact
        assert np.all((f >= 0) & (f <= 1))
        if acc:
            err = np.abs(f[learned] - ex_f[learned])
            assert err.mean() < 0.15
        fallbacks.append(fb)
    assert fallbacks[0] <= fallbacks[1] <= fallbacks[2]
    # the hard shadow never changes: BOTH jobs keep bit-identical silhouettes
    both_exact, _ = run(None, 0.0, 3)
    both_net, _ = run(net, 0.1, 3)
    assert torch.equal(both_exact.vis_silhouette, both_net.vis_silhouette)
    assert torch.equal(both_exact.vis_filter, both_net.vis_filter)


def test_what_the_trained_network_gains(lib):
    """On held-out edge fragments, with every surrogate answer accepted (no
    guard), the trained network's mean error against the exact RSMSS answer
    is well below that of the untrained network and below that of the hard
    shadow test alone (the method without any penumbra estimate); the guard
    (other tests) then sends the doubtful ones to the exact walk."""
    api, S = lib
    import rbsm_scenes as sc
    train = [sc.config2(s, screen=(1280, 720)) for s in (20, 21)]
    data = [(dev(f.depth), dev(f.x), dev(f.y), dev(f.z)) for f in train]
    samples, count = S.Surrogate.dataset(data, capacity=1 << 20)
    untrained = S.Surrogate(sc.mlp_init(0))
    trained = S.Surrogate(sc.mlp_init(0))
    trained.train(samples, count, epochs=4, batch=4096, lr=3e-3)
    test = sc.config2(22, screen=(1280, 720))
    depth, x, y, z = dev(test.depth), dev(test.x), dev(test.y), dev(test.z)

    def run(surrogate):
        job = api.Job(0, x, y, z, mode=2, codes=True)
        b = api.Batch([depth], [job], surrogate=surrogate, guard_tau=1e6 if surrogate else 0.0)
        api.rbsm_batch_run(b)
        torch.cuda.synchronize()
        return job.vis_filter.cpu().numpy().astype(np.float64), job.codes.cpu().numpy().view(np.uint16)

    exact, codes = run(None)
    edge = ((codes >> 9) & 1) == 1
    assert edge.sum() > 1000
    hard = 1.0 - ((codes >> 4) & 1).astype(np.float64)          # the shadow test alone (1 = lit)
    answers, answered = {}, edge.copy()
    for name, net in (("untrained", untrained), ("trained", trained)):
        f, c = run(net)
        answered &= ((c >> 10) & 1) == 1                          # answered by the network
        answers[name] = f
    assert answered.sum() > 0.9 * edge.sum()
    err = {name: np.abs(f[answered] - exact[answered]).mean() for name, f in answers.items()}
    err["hard"] = np.abs(hard[answered] - exact[answered]).mean()
    # measured on this scene: untrained 0.42, trained 0.12, hard 0.16
    assert err["trained"] < 0.5 * err["untrained"], err
    assert err["trained"] < 0.85 * err["hard"], err
