"""Autotuner bookkeeping (host only): size classes, table lookup and option application."""
import json

import pytest

from ._util import ensure_built


@pytest.fixture(scope="module")
def B():
    ensure_built()
    from paper_2311_12134_gb300 import binding
    return binding


def test_size_classes_bucket_n_and_units():
    from paper_2311_12134_gb300 import autotune as at
    assert at.size_class("GB300", "mixed", 3, 944, 11880) == "GB300|mixed|lmax3|n<=1024|units<=65536"
    assert at.size_class("GB300", "mixed", 3, 688, 512) == "GB300|mixed|lmax3|n<=768|units<=1024"
    assert at.size_class("GB300", "fp64", 3, 2192, 31840) == "GB300|fp64|lmax3|n<=3072|units<=65536"
    assert at.size_class("GB300", "mixed", 3, 99999, 1 << 29).endswith("n<=16384|units<=1073741824")


def test_candidates_cover_the_defaults_and_are_valid_options(B):
    from paper_2311_12134_gb300 import autotune as at
    cands = at.candidates()
    assert at.DEFAULTS in cands and len({json.dumps(c, sort_keys=True) for c in cands}) == len(cands)
    saved = {k: B.get_option(k) for k in at.DEFAULTS}
    try:
        for c in cands:            # every candidate is accepted by lsms_set_option
            at.apply(c)
            assert all(B.get_option(k) == v or (k == "streams" and v == 0) for k, v in c.items())
    finally:
        at.apply(saved)


def test_table_lookup(tmp_path):
    from paper_2311_12134_gb300 import autotune as at

    class FakeLiz:
        max_sites = 59

    class FakeProblem:
        K = 16
        lmax = 3
        precision = "mixed"
        n_units = 11880
        liz = FakeLiz()
        device = None

    table = {"X|mixed|lmax3|n<=1024|units<=65536": {"settings": {"solve_cols": 16, "solve_regs": 1, "streams": 4}}}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(table))
    import paper_2311_12134_gb300.autotune as mod
    orig = mod.problem_class
    try:
        mod.problem_class = lambda p: at.size_class("X", p.precision, p.lmax, p.K * p.liz.max_sites, p.n_units)
        assert at.lookup(FakeProblem(), path=str(path)) == {"solve_cols": 16, "solve_regs": 1, "streams": 4}
        FakeProblem.n_units = 100
        assert at.lookup(FakeProblem(), path=str(path)) is None
    finally:
        mod.problem_class = orig
