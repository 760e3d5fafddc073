"""The k-distance merge's argument, checked on a model (no GPU): each point's
screened squared distance s is off its true value by at most E (the
screen's bound for that pair of rows); every part of the cloud keeps the 8
smallest lower bounds l = s - E; U is the k-th smallest upper bound l + 2E
over those lists; a list whose last entry exceeds U holds every point of its
part with l <= U, and the other parts are taken whole. The k-th smallest true
value is then always among the candidates. Errors are drawn adversarially
(at the bound, either sign) and with many exact ties."""
import numpy as np
import pytest

L = 8                                            # entries per list, as on the tensor cores


def _merge_model(true, E, parts, k, far=False):
    key_true = -true if far else true
    rng = np.random.default_rng(len(true) + k)
    # screened keys within +-E of the true keys, often at the bound
    sign = rng.choice([-1.0, 1.0, 0.0], size=true.size, p=[0.4, 0.4, 0.2])
    s = key_true + sign * E
    lo = s - E
    lists = []
    for p in parts:
        order = p[np.argsort(lo[p], kind="stable")][:L]
        lists.append((p, order))
    ub = [lo[j] + 2 * E[j] for _, order in lists for j in order]
    U = np.sort(ub)[k - 1]
    cand = []
    for p, order in lists:
        if order.size == L and not lo[order[-1]] > U:
            cand.extend(p.tolist())              # part taken whole
        else:
            cand.extend([j for j in order if lo[j] <= U])
    cand = np.unique(cand)
    got = np.sort(key_true[cand])[k - 1]
    want = np.sort(key_true)[k - 1]
    return got, want, cand.size


@pytest.mark.parametrize("far", [False, True])
@pytest.mark.parametrize("seed", range(40))
def test_merge_model_finds_the_kth(seed, far):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    # clustered values with exact ties, and bounds of different sizes per point
    true = np.round(rng.gamma(2.0, 50.0, size=n) * 4) / 4
    if seed % 3 == 0:
        true[rng.integers(0, n, size=n // 3)] = true[0]
    E = rng.uniform(0.0, 6.0, size=n) * (seed % 4 != 0)
    n_parts = int(rng.integers(1, 40))
    cut = np.sort(rng.choice(np.arange(1, n), size=min(n_parts - 1, n - 1), replace=False)) if n > 1 else []
    parts = [p for p in np.split(rng.permutation(n), cut) if p.size]
    for k in (1, 2, 5, min(8, n)):
        if k > n:
            continue
        got, want, _ = _merge_model(true, E, parts, k, far)
        assert got == want, (seed, k, far)


def test_merge_model_candidates_stay_few_when_bounds_are_tight():
    rng = np.random.default_rng(7)
    n = 20000
    true = rng.normal(500.0, 40.0, size=n)
    E = np.full(n, 0.5)
    parts = np.array_split(rng.permutation(n), 64)
    got, want, n_cand = _merge_model(true, E, parts, 5)
    assert got == want and n_cand < 100


def _sampled_model(true, E, sample, k, cap, far=False):
    """The sampled-threshold flow: tau = the k-th smallest upper bound l + 2E
    over the sample's lists (here: the whole sample, which only tightens
    tau); the full screen keeps every point with l <= tau (a query with more
    than cap of them would take the list screen); U = the k-th smallest
    upper bound over those; the candidates are the kept points with l <= U."""
    key_true = -true if far else true
    rng = np.random.default_rng(len(true) + 3 * k)
    sign = rng.choice([-1.0, 1.0, 0.0], size=true.size, p=[0.4, 0.4, 0.2])
    lo = key_true + sign * E - E
    ub = lo + 2 * E
    tau = np.sort(ub[sample])[k - 1]
    kept = np.nonzero(lo <= tau)[0]
    if kept.size > cap:
        return None, np.sort(key_true)[k - 1], kept.size
    U = np.sort(ub[kept])[k - 1]
    cand = kept[lo[kept] <= U]
    return np.sort(key_true[cand])[k - 1], np.sort(key_true)[k - 1], kept.size


@pytest.mark.parametrize("far", [False, True])
@pytest.mark.parametrize("seed", range(30))
def test_sampled_threshold_model_finds_the_kth(seed, far):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 4000))
    true = np.round(rng.gamma(2.0, 50.0, size=n) * 4) / 4
    if seed % 3 == 0:
        true[rng.integers(0, n, size=n // 3)] = true[0]
    E = rng.uniform(0.0, 6.0, size=n) * (seed % 4 != 0)
    stride = int(rng.integers(1, 40))
    sample = np.arange(0, n, stride)
    for k in (1, 2, 5, 8):
        if k > sample.size:
            continue
        got, want, kept = _sampled_model(true, E, sample, k, cap=n, far=far)
        assert got == want, (seed, k, far)
        assert kept >= k


def _interval_model(exact, eta, tiny, k, far=False):
    """The merge's last step: FP32 values f with |f - d2| <= eta d2 + tiny
    (adversarial, at the bound), keys g (d2, or -d2 far); Gk the k-th
    smallest g; klo / khi the key interval of a value; candidates with
    khi < klo(Gk) are below the k-th exact key (nb of them), those with klo
    > khi(Gk) above it; the k-th exact key is the (k - nb)-th of the rest."""
    rng = np.random.default_rng(exact.size + k)
    sgn = rng.choice([-1.0, 1.0, 0.0], size=exact.size, p=[0.4, 0.4, 0.2])
    f = exact + sgn * (eta * exact + tiny)
    d2_lo = (f - tiny) / (1 + eta)
    d2_hi = (f + tiny) / (1 - eta)
    g = -f if far else f
    klo = -d2_hi if far else d2_lo
    khi = -d2_lo if far else d2_hi
    order = np.argsort(g, kind="stable")
    gk_i = order[k - 1]
    t_lo, t_hi = klo[gk_i], khi[gk_i]
    below = khi < t_lo
    mid = ~below & ~(klo > t_hi)
    nb = int(below.sum())
    key = -exact if far else exact
    assert nb <= k - 1 and mid.sum() >= k - nb
    got = np.sort(key[mid])[k - nb - 1]
    return got, np.sort(key)[k - 1], int(mid.sum())


@pytest.mark.parametrize("far", [False, True])
@pytest.mark.parametrize("seed", range(30))
def test_interval_model_settles_the_kth(seed, far):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(1, 500))
    exact = np.round(rng.gamma(2.0, 30.0, size=n) * 8) / 8
    if seed % 3 == 0:
        exact[rng.integers(0, n, size=n // 2)] = exact[0]
    eta = [1e-6, 1e-4, 1e-2][seed % 3]
    for k in (1, 2, 5, 8):
        if k > n:
            continue
        got, want, _ = _interval_model(exact, eta, 1e-30, k, far)
        assert got == want, (seed, k, far)


def test_interval_model_leaves_one_candidate_when_values_are_apart():
    rng = np.random.default_rng(9)
    exact = np.sort(rng.uniform(100.0, 200.0, size=300))
    got, want, n_mid = _interval_model(exact, 2.3e-5, 1e-40, 5)
    assert got == want and n_mid == 1
