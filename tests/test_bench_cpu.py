"""Host logic of bench.py that feeds the roofline fields (no GPU)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_measured_traffic_follows_the_source_it_was_taken_on(monkeypatch):
    # the committed capture belongs to the committed local-solve source
    b = bench.measured_traffic("local_solve", "local_solve.cu")
    assert b is not None and b > 0
    # any other source: no traffic figure (the bench line then prints null)
    entry = dict(bench.MEASURED_TRAFFIC["local_solve"])
    entry["source_sha256"] = "0" * 64
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "local_solve", entry)
    assert bench.measured_traffic("local_solve", "local_solve.cu") is None
    assert bench.measured_traffic("no_such_phase", "local_solve.cu") is None


def _levels(scale):
    return [
        {"n": 1000 * scale, "nc": 300 * scale, "nnz": 5000 * scale, "nnz_R": 2000 * scale,
         "nnz_P": 2500 * scale},
        {"n": 300 * scale, "nc": 0, "nnz": 2400 * scale},
    ]


def test_phase_bytes_scale_with_the_level_sizes():
    one, two, three = (bench.phase_bytes(_levels(c)) for c in (1, 2, 3))
    assert set(one) == {"split", "pattern", "weight", "smooth", "galerkin"}
    for k in one:
        assert one[k] > 0
        # every term is affine in the sizes (the row pointers' n + 1 entries)
        assert three[k] - two[k] == two[k] - one[k], k
        assert two[k] > one[k], k


def test_levels_without_transfers_cost_nothing():
    coarsest = [{"n": 50, "nc": 0, "nnz": 400}]
    assert all(v == 0.0 for v in bench.phase_bytes(coarsest).values())


def test_galerkin_bytes_read_every_operand_once():
    b = bench.phase_bytes(_levels(1))["galerkin"]
    # R, A, P read and A_c written once: at least 12 bytes per stored entry of each
    assert b >= 12 * (2000 + 5000 + 2500 + 2400)
