"""The long-run conservation tool on a short run: every form and precision runs, the
spectral-resident FP64 run is the reference, and the drifts are at their precision's level."""
import pytest

pytestmark = pytest.mark.gpu


def test_drift_report_short_run():
    from paper_2210_06232_gb300 import drift

    rows = drift.run(n=16, steps=200, h=0.1, every=20, seed=3, sigma=4.0)
    assert [(r["precision"], r["form"]) for r in rows] == [
        ("fp64", "spectral"), ("fp64", "literal"), ("fp64", "xy"), ("fp32", "spectral"), ("fp32", "literal"),
        ("fp32", "xy")]
    by = {(r["precision"], r["form"]): r for r in rows}
    assert all(r["records"] == 11 for r in rows)
    assert by[("fp64", "spectral")]["fields_rel_l2_vs_fp64_spectral"] == 0.0
    assert by[("fp64", "spectral")]["E1_rel_drift"] < 1e-14
    for form in ("literal", "xy"):
        assert by[("fp64", form)]["E1_rel_drift"] < 1e-13
        assert by[("fp64", form)]["fields_rel_l2_vs_fp64_spectral"] < 1e-12
    for form in ("spectral", "literal", "xy"):
        assert by[("fp32", form)]["E1_rel_drift"] < 1e-5
        assert by[("fp32", form)]["fields_rel_l2_vs_fp64_spectral"] < 1e-5
