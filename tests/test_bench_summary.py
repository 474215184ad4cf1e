"""The bench line's closing summary (host logic, no GPU): built from a
synthetic line with the sections the default run fills, it ends with the
mixed-precision digest the metric asks for -- per precision the speed-up over
the FP64 step and, per variable, the L2 and max errors against the exact
solution and against the FP64 result -- and the step-level roofline picks the
largest term."""
import json

import pytest


def _line():
    names = ["rho", "rho_u", "rho_v", "rho_w", "E"]

    def entry(x, err, vs):
        e = {"value": 5.86e8 * x, "l2_rel_err_vs_exact": {v: err for v in names},
             "max_rel_err_vs_exact": {v: 10 * err for v in names},
             "step_roofline": {"bound": "fp64_alu", "frac": 0.85}}
        if vs is not None:
            e["speedup_vs_fp64"] = x
            e["vs_fp64_per_var"] = {v: {"rel_l2": vs, "rel_max": 10 * vs} for v in names}
        return e

    mixed = {"df64": entry(3.08, 1.7e-11, 3.4e-15), "fp32": entry(12.5, 1.9e-8, 7.4e-8),
             "fp64": entry(1.0, 1.7e-11, None), "note": "predictor arithmetic"}
    return {"value": 5.86e8, "remesh": {"ms_each": [26.0]}, "mixed": mixed,
            "configs": {"euler3d-n7-amr": {"fp64": entry(1.0, 1.6e-13, None), "workload": "n7"},
                        "euler2d-n3-vortex": entry(1.0, 2.9e-6, None)},
            "dd_virtual": {"overhead": 0.003},
            "shifted_fixed_dt": {"fp64": {"speedup_vs_ader_step": 1.01}, "workload": "w"}}


def test_summary_ends_with_the_mixed_digest():
    import bench
    s = bench.summarise(_line())
    assert list(s)[-1] == "mixed_summary"
    ms = s["mixed_summary"]
    assert ms["vars"] == ["rho", "rho_u", "rho_v", "rho_w", "E"]
    assert ms["df64"]["x"] == 3.08 and ms["fp32"]["x"] == 12.5 and ms["fp64"]["x"] == 1.0
    assert ms["df64"]["exact_l2"] == [1.7e-11] * 5 and ms["df64"]["exact_max"] == [1.7e-10] * 5
    assert ms["fp32"]["vs64_l2"] == [7.4e-8] * 5 and ms["fp32"]["vs64_max"] == [7.4e-7] * 5
    assert ms["fp64"]["vs64_l2"] is None
    assert "note" not in ms
    assert s["shifted_x"] == {"fp64": 1.01}
    assert s["n5"]["df64"]["x"] == 3.08 and s["n7"]["fp64"]["err_rho"] == 1.6e-13
    json.dumps(s)                                  # serialisable as the line's tail


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32", "tf32x3"])
def test_step_roofline_binds_the_largest_term(prec):
    import bench
    r = bench.step_roofline(prec, 3, 5, 5, 268087, 0.5)
    terms = r["terms_ms"]
    assert r["bound"] == max(terms, key=terms.get)
    assert abs(r["frac"] - terms[r["bound"]] / 500.0) < 1e-12
    if prec == "fp64":
        # the FP64 step is bound by the FP64 ALU: predictor + faces + corrector flops
        assert r["bound"] == "fp64_alu" and terms["fp64_alu"] > 100 * terms["hbm"]
