"""The seeded input recipe: deterministic, in range, and a valid candidate CSR."""
import numpy as np

import instances as I

# fingerprints of the point sets; a change here means the recipe changed
SHA = {
    ("uniform", 1000, 0): "50370ae24cb8e28eea7133ced2a7689e2e501199e07944c75cfea09a836c7334",
    ("mixture", 1000, 0): "676b5dd4c0287a9d86bb7d15eab8104ec2d5f0fe3b3fd324c7cb12e6a20acfbc",
    ("uniform", 100000, 0): "8312ef928e01c1cdbfa96e9e74af131076ef754ff97a8e1d6a1e14b730295d36",
    ("mixture", 200000, 0): "1b4f2e040bdb412740295d2b4b6936690fee46aa015d1f261824f4e48f459404",
}


def test_point_fingerprints():
    for (kind, n, seed), h in SHA.items():
        xy = I.uniform_points(n, seed) if kind == "uniform" else I.mixture_points(n, seed)
        assert I.points_sha256(xy) == h, (kind, n, seed)


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    out = I.draws(np.uint64(0), 0, 3)
    assert [hex(int(x)) for x in out] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4", "0x6c45d188009454f"]


def test_points_deterministic_and_in_box():
    for kind in ("uniform", "mixture"):
        a = I.make_instance(kind, 1000, 0, 10)
        b = I.make_instance(kind, 1000, 0, 10)
        assert a["sha256"] == b["sha256"]
        assert a["xy"].min() >= 0 and a["xy"].max() <= 1_000_000
        assert a["sha256"] != I.make_instance(kind, 1000, 1, 10)["sha256"]


def test_normal_deviates_moments():
    g = I.normal_deviates(I.stream_key(0, I.TAG_NORMAL), np.arange(200000))
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01 and np.abs(g).max() <= 6


def test_knn_csr_valid_and_exact():
    xy = I.mixture_points(3000, 2)
    rp, col = I.knn_csr(xy, 10)
    n = 3000
    src = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(np.diff(rp) >= 10)
    assert np.all(src != col)
    for v in range(n):  # sorted, no duplicates
        r = col[rp[v]:rp[v + 1]]
        assert np.all(np.diff(r) > 0)
    pairs = set(zip(src.tolist(), col.tolist()))
    assert all((b, a) in pairs for a, b in pairs)
    # brute-force k nearest (d2, index) for a sample of nodes are all present
    for u in range(0, n, 97):
        d = xy.astype(np.int64) - xy[u]
        d2 = d[:, 0] ** 2 + d[:, 1] ** 2
        key = d2 * n + np.arange(n)
        key[u] = np.iinfo(np.int64).max
        nn = np.argsort(key)[:10]
        assert all((u, int(w)) in pairs for w in nn)
