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
from tests import mlp_bounds as mb  # noqa: E402
from tests.test_gpu_parity import dev  # noqa: E402
from tests.window_rule import walks_inside_window  # noqa: E402


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


def test_forward_matches_reference(lib, scene):
    """Every output within the element-wise bound of tests/mlp_bounds.py
    (FP32 accumulation, and BF16 rounding or ReLU decisions that the
    accumulation difference can flip); ragged tile counts included."""
    api, S = lib
    import rbsm_scenes as sc
    feat, labels = _oracle_samples(scene)
    P32 = sc.mlp_init(1)
    net = S.Surrogate(P32)
    P = {k: v.astype(np.float64) for k, v in P32.items()}
    for n in (labels.size, 1, 127, 129, 1000):
        f = {k: v[:n] for k, v in feat.items()}
        samples, m = S.Surrogate.pack(f, labels[:n])
        out = net.forward(samples, m).cpu().numpy().astype(np.float64)
        c = mb.forward_intervals(P, omlp.encode(f))
        assert np.all(np.abs(out - c["y"]) <= c["d_y"]), (n, np.max(np.abs(out - c["y"]) - c["d_y"]))


def _grad_case(S, feat, labels, n, seed):
    import rbsm_scenes as sc
    f = {k: v[:n] for k, v in feat.items()}
    P32 = sc.mlp_init(seed)
    net = S.Surrogate(P32)
    samples, m = S.Surrogate.pack(f, labels[:n])
    order = torch.arange(m, dtype=torch.int32, device="cuda")
    P = {k: v.astype(np.float64) for k, v in P32.items()}
    return net, samples, order, P, omlp.encode(f), labels[:n]


def _assert_within(got, ref, bound, what):
    d = np.abs(got - ref)
    bad = d > bound
    assert not np.any(bad), (what, int(bad.sum()), float(np.max(d - bound)))


@pytest.mark.parametrize("n", [4096, 1000])
def test_gradient_and_adam_match_reference_element_wise(lib, scene, n):
    """Every gradient entry, the loss and every parameter after one Adam step
    within the element-wise bounds of tests/mlp_bounds.py."""
    api, S = lib
    feat, labels = _oracle_samples(scene)
    net, samples, order, P, X, t = _grad_case(S, feat, labels, n, 2)
    net.grad(samples, order)
    g = S.Surrogate.unflatten(net.read_grad())
    loss_gpu = net.take_loss() / n
    loss, loss_bound, G, bound = mb.gradient_bounds(P, X, t)
    assert abs(loss_gpu - loss) <= loss_bound
    for k in G:
        _assert_within(g[k], G[k], bound[k], k)
    net.adam(1e-3)
    after = S.Surrogate.unflatten(net.params())
    Pn, dev = mb.adam_first_step_bounds(P, G, bound, 1e-3)
    for k in P:
        _assert_within(after[k], Pn[k], dev[k], "adam " + k)


def test_gradient_over_many_tiles_per_cta(lib):
    """A batch of 300 tiles and a ragged tail: 256 CTAs, some summing two
    tiles in tensor memory before writing their partials."""
    api, S = lib
    rng = np.random.Generator(np.random.PCG64(5))
    n = 128 * 300 + 37
    feat = {"bits": rng.integers(0, 1 << 25, n, dtype=np.uint64).astype(np.uint32),
            "fx": rng.random(n, dtype=np.float32), "fy": rng.random(n, dtype=np.float32),
            "gap": (rng.random(n, dtype=np.float32) * 0.3).astype(np.float32)}
    labels = rng.random(n).astype(np.float32)
    net, samples, order, P, X, t = _grad_case(S, feat, labels, n, 4)
    perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    net.grad(samples, perm)
    g = S.Surrogate.unflatten(net.read_grad())
    loss, loss_bound, G, bound = mb.gradient_bounds(P, X, t)     # order does not change the sum
    assert abs(net.take_loss() / n - loss) <= loss_bound
    for k in G:
        _assert_within(g[k], G[k], bound[k], k)


def test_training_step_is_reproducible_and_equals_grad_then_adam(lib, scene):
    """Fixed-order reductions: the same minibatch gives the same gradient
    bits twice, and the fused step (reduction + Adam in one kernel) gives the
    bits of rbsm_mlp_grad followed by rbsm_mlp_adam."""
    api, S = lib
    feat, labels = _oracle_samples(scene)
    a, samples, order, *_ = _grad_case(S, feat, labels, 4096, 6)
    b, *_ = _grad_case(S, feat, labels, 4096, 6)
    a.grad(samples, order)
    g1 = a.read_grad()
    a.grad(samples, order)
    g2 = a.read_grad()
    assert np.array_equal(2 * g1, g2)                                 # exact: x + x = 2x
    a.load(S.Surrogate.unflatten(b.params()))
    for step in range(3):
        a.grad(samples, order)
        a.adam(2e-3)
        b.train_step(samples, order, 2e-3)
    assert np.array_equal(a.params(), b.params())
    assert a.take_loss() == b.take_loss()


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
    """On held-out edge fragments whose walks stop inside the window (the
    only ones the structural guard lets the network answer), with every
    such answer accepted (no error-estimate guard), the trained network's
    mean error against the exact RSMSS answer is well below that of the
    untrained network and of the hard shadow test alone (the method without
    any penumbra estimate)."""
    api, S = lib
    import rbsm_scenes as sc
    train = [sc.config2(s, screen=(1280, 720)) for s in (20, 21)]
    data = [(dev(f.depth), dev(f.x), dev(f.y), dev(f.z)) for f in train]
    samples, count = S.Surrogate.dataset(data, capacity=1 << 20, in_window=True)
    untrained = S.Surrogate(sc.mlp_init(0))
    trained = S.Surrogate(sc.mlp_init(0))
    trained.train(samples, count, epochs=30, batch=1024, lr=3e-3, lr_decay=0.9)
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
    feat = orc.features(test.depth, test.x[edge], test.y[edge], test.z[edge])
    inside = np.zeros_like(edge)
    inside[edge] = walks_inside_window(feat["bits"])
    assert inside.sum() > 1000
    hard = 1.0 - ((codes >> 4) & 1).astype(np.float64)          # the shadow test alone (1 = lit)
    answers = {}
    for name, net in (("untrained", untrained), ("trained", trained)):
        f, c = run(net)
        answered = ((c >> 10) & 1) == 1
        assert np.array_equal(answered, inside)                   # the structural guard, fragment by fragment
        answers[name] = f
    err = {name: np.abs(f[inside] - exact[inside]).mean() for name, f in answers.items()}
    err["hard"] = np.abs(hard[inside] - exact[inside]).mean()
    assert err["trained"] < 0.3 * err["untrained"], err
    assert err["trained"] < 0.3 * err["hard"], err


# The surrogate's stated error bound: over the edge fragments it answers
# with the committed checkpoint (its trusted-pattern bitmap in force) and
# guard_tau = 0.01, the absolute error against the exact Listing 5 answer
# has mean <= 0.01, 99th percentile <= 0.03 and maximum <= 0.1.  The bound
# and tau were chosen on C2 seeds 12, 22, 31 and C4 seed 100 (largest error
# 0.069); the scenes below served neither that nor training (C4 seeds
# 0-114) nor calibration (C4 seeds 115-235).
BOUND_TAU = 0.01
BOUND = {"mean": 0.01, "p99": 0.03, "max": 0.1}


@pytest.mark.parametrize("recipe", ["C2 seed 41", "C4 seed 102"])
def test_surrogate_meets_its_stated_bound_on_held_out_scenes(lib, recipe):
    api, S = lib
    import os
    import rbsm_scenes as sc
    f = sc.config2(41) if recipe.startswith("C2") else sc.config4(102)
    net = S.Surrogate.from_checkpoint(os.path.join(os.path.dirname(S.__file__), "weights", "surrogate_c4.npz"))
    assert net.trust is not None
    depth, x, y, z = dev(f.depth), dev(f.x), dev(f.y), dev(f.z)
    job = api.Job(0, x, y, z, mode=2, codes=True)
    b = api.Batch([depth], [job], surrogate=net, guard_tau=BOUND_TAU)
    api.rbsm_batch_run(b)
    torch.cuda.synchronize()
    acc, fb = api.rbsm_batch_surrogate_counts(b)
    codes = job.codes.cpu().numpy().view(np.uint16)
    vis = job.vis_filter.cpu().numpy().astype(np.float64)
    answered = ((codes >> 10) & 1) == 1
    assert answered.sum() == acc > 10000
    # reference answers: the oracle's Listing 5 answer of every answered fragment
    ref = orc.evaluate(f.depth, f.x[answered], f.y[answered], f.z[answered], orc.MODE_FILTER)
    assert np.all(((ref["codes"] >> 9) & 1) == 1)                  # only edge fragments are answered
    feat = orc.features(f.depth, f.x[answered], f.y[answered], f.z[answered])
    assert np.all(walks_inside_window(feat["bits"]))              # only inside-window ones
    p = feat["bits"].astype(np.uint32)
    assert np.all((net.trust[p >> 5] >> (p & 31)) & 1)            # only trusted patterns
    err = np.abs(vis[answered] - ref["vis"])
    got = {"mean": err.mean(), "p99": np.quantile(err, 0.99), "max": err.max()}
    assert all(got[k] <= BOUND[k] for k in BOUND), (got, acc, fb)


@pytest.mark.parametrize("limit_ns", [20_000, 2_000_000])
def test_bounded_wait_gives_up_instead_of_hanging(lib, limit_ns):
    """The mbarrier wait every tensor-core kernel uses gives up after its
    limit on a barrier that nothing arrives at (so a lost completion becomes
    RBSM_ERR_TIMEOUT, not a hung GPU), completes once the barrier has its
    arrival, and the context stays usable afterwards."""
    api, _ = lib
    gave_up, completed, waited = api.rbsm_selftest_bounded_wait(limit_ns)
    assert gave_up and completed
    assert limit_ns <= waited < limit_ns + 100_000_000
    t = torch.arange(8, device="cuda", dtype=torch.float32)
    assert float(t.sum()) == 28.0
