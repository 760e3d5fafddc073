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
