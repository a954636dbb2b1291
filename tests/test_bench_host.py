"""Host-side helpers of bench.py (no GPU): the algorithmic FLOP model of the
warm-start network, the oracle-error field of the bench line and the
recorded-traffic gate."""
import numpy as np

import bench


def test_fno_flop_model_scales_as_written():
    # doubling the grid multiplies the N^3 terms by 8 and the N^2 / N terms
    # by less: the ratio lies strictly between 4 and 8
    a = bench.fno_flops_per_sample(32, 12, 4)
    b = bench.fno_flops_per_sample(64, 12, 4)
    assert 4 < b["forward"] / a["forward"] < 8
    assert b["train"] > 2 * b["forward"]
    # layers enter linearly (the head is counted once per pass)
    one, two = bench.fno_flops_per_sample(64, 12, 1), bench.fno_flops_per_sample(64, 12, 2)
    head_fwd = 2 * 64 ** 3 * (36 * 16 + 36)
    assert two["forward"] - head_fwd == 2 * (one["forward"] - head_fwd)


def test_oracle_error_against_the_stored_solve():
    import json
    import os
    ref = json.load(open(os.path.join(bench.ROOT, "tests", "golden",
                                      "softincl128_warm_oracle_solve.json")))["mean_stress"]
    got = np.array(ref) * (1 + 1e-6)
    e = bench.oracle_error("warm", got)
    assert e is not None and abs(e["mean_stress_max_rel"] - 1e-6) < 1e-9


def test_recorded_traffic_is_gated_by_the_kernel_sources():
    # the record matches the current sources (it is re-keyed with every capture)
    assert bench.recorded_traffic("gamma_apply_128") is not None
    assert bench.recorded_traffic("polarization_map_128") is not None
    assert bench.recorded_traffic("no_such_kernel") is None


def test_cold_form_error_falls_back_to_the_same_fixed_point():
    """Without a stored cold-form oracle solve, the cold form is compared with
    the oracle's warm-form solve of the same cell (same fixed point of F)."""
    import json
    import os
    ref = json.load(open(os.path.join(bench.ROOT, "tests", "golden",
                                      "softincl128_warm_oracle_solve.json")))["mean_stress"]
    e = bench.oracle_error("cold", ref)
    assert e is not None and e["mean_stress_max_rel"] == 0.0
    assert e["reference"].endswith(".json")
