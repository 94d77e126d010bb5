"""TSPLIB reader (host code of the C ABI; no GPU needed) and, on the GPU, the
Section 5.1 program that solves a TSPLIB problem end to end."""
import numpy as np
import pytest

import instances as I
import paper_2011_08170_gb300 as f2m
from paper_2011_08170_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return f2m.load()


def to_tsplib(xy, name="synthetic", ids=None):
    ids = np.arange(1, len(xy) + 1) if ids is None else ids
    lines = [f"NAME : {name}", "TYPE : TSP", f"DIMENSION : {len(xy)}", "EDGE_WEIGHT_TYPE : EUC_2D",
             "NODE_COORD_SECTION"]
    lines += [f"{i} {x} {y}" for i, (x, y) in zip(np.asarray(ids).tolist(), np.asarray(xy).tolist())]
    return "\n".join(lines + ["EOF", ""])


HAND = "\n".join([
    "NAME: tiny",
    "COMMENT : four points, written by hand",
    "TYPE TSP",
    "DIMENSION: 4",
    "EDGE_WEIGHT_TYPE EUC_2D",
    "NODE_COORD_SECTION",
    "3 12.0 -7",
    "1 1.2e1 3",
    "4 -5 0.0",
    "2 100 40",
    "EOF",
    ""])


def test_parse_forms_order_and_translation(lib):
    xy, tr = f2m.f2m_tsplib_parse(HAND)
    assert tr == (-5, -7)
    assert xy.tolist() == [[17, 10], [105, 47], [17, 0], [0, 7]]


HEAD = "DIMENSION: 2\nEDGE_WEIGHT_TYPE: EUC_2D\n"


@pytest.mark.parametrize("text,why", [
    ("DIMENSION: 2\nEDGE_WEIGHT_TYPE: GEO\nNODE_COORD_SECTION\n1 0 0\n2 1 1\n", "EUC_2D only"),
    ("EDGE_WEIGHT_TYPE: EUC_2D\nNODE_COORD_SECTION\n1 0 0\n", "DIMENSION must come"),
    ("DIMENSION: 3\nEDGE_WEIGHT_TYPE: EUC_2D\nNODE_COORD_SECTION\n1 0 0\n2 1 1\n", "has 2 nodes"),
    (HEAD + "NODE_COORD_SECTION\n1 0 0\n1 1 1\n", "repeated"),
    (HEAD + "NODE_COORD_SECTION\n1 0 0.5\n2 1 1\n", "integral"),
    (HEAD + "NODE_COORD_SECTION\n1 0 0\n2 2000000 1\n", "spread"),
    ("TYPE: ATSP\n" + HEAD + "NODE_COORD_SECTION\n1 0 0\n2 1 1\n", "TSP only"),
    (HEAD + "EDGE_WEIGHT_SECTION\n0 1\n", "not supported"),
    (HEAD + "NODE_COORD_SECTION\n3 0 0\n2 1 1\n", "out of 1..DIMENSION"),
    (HEAD, "no NODE_COORD_SECTION"),
])
def test_parse_rejects(lib, text, why):
    with pytest.raises(f2m.F2MError) as ei:
        f2m.f2m_tsplib_parse(text)
    assert ei.value.status == f2m.F2M_ERR_INVALID_ARG and why in str(ei.value)


def test_round_trip_shuffled_ids(lib):
    d = I.make_instance("mixture", 5000, 4, 10)
    perm = np.random.default_rng(0).permutation(5000)
    text = to_tsplib(d["xy"][perm], ids=perm + 1)  # lines in a shuffled order
    xy, tr = f2m.f2m_tsplib_parse(text)
    lo = d["xy"].min(axis=0)
    assert tr == (int(lo[0]), int(lo[1]))
    assert np.array_equal(xy, d["xy"] - lo)


@pytest.mark.gpu
def test_program_solves_a_tsplib_file(lib, oracle_lib, tmp_path):
    from paper_2011_08170_gb300 import solve_tsp
    d = I.make_instance("uniform", 3000, 9, 10)
    path = tmp_path / "u3000.tsp"
    path.write_text(to_tsplib(d["xy"] + 12345))
    out = tmp_path / "u3000.sol"
    assert solve_tsp.main([str(path), "-k", "10", "-o", str(out)]) == 0
    xy, info, edges, x2 = solve_tsp.solve_file(str(path), 10)
    rp, col = oracle_lib.knn_csr(xy, 10)
    r = oracle_lib.solve(xy, rp, col)
    assert info["certified"] == 2 and r.certified == 2
    assert info["bound2"] << (9 - info["frac_bits"]) == r.bound2 << (9 - r.frac_bits)
    # the written solution: every node's x sums to 2, and its cost is the optimum
    rows = [ln.split() for ln in out.read_text().splitlines() if not ln.startswith("#")]
    u = np.array([int(a) - 1 for a, _, _ in rows])
    v = np.array([int(b) - 1 for _, b, _ in rows])
    x = np.array([float(c) for _, _, c in rows])
    assert np.allclose(np.bincount(u, x, 3000) + np.bincount(v, x, 3000), 2.0)
    dd = (xy[u] - xy[v]).astype(np.float64)
    c = np.floor(np.sqrt(dd[:, 0] ** 2 + dd[:, 1] ** 2) + 0.5)
    assert abs((c * x).sum() - r.opt) < 1e-6
