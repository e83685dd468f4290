"""The chain-step counts behind the policy partition (balanced by the sum of
S_p) and behind the benchmark's algorithmic operation count (3 flop per
one-state chain-step, 16 per reversionary chain-step) are the oracle's own
projection lengths, for every product and with a horizon."""
import numpy as np
import pytest

import oracle
import synth
from paper_1401_1757_gb300.shard import projection_steps


@pytest.mark.parametrize("horizon", [0, 1, 333, 600])
def test_projection_steps_match_the_oracle(horizon):
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(3000, seed=17)
    S = projection_steps(pol, n_ages=len(tab), horizon=horizon)
    for i in range(len(pol["product"])):
        So, _ = oracle.steps(int(pol["product"][i]), int(pol["age1_m"][i]), int(pol["age2_m"][i]),
                             int(pol["term_m"][i]), len(tab), horizon)
        assert S[i] == So, (i, int(pol["product"][i]), S[i], So)


def test_bench_algorithmic_count():
    """3 flop per one-state chain-step and 16 per reversionary chain-step,
    times the scenarios."""
    import sys
    sys.argv = ["bench.py"]
    import bench
    pol = synth.portfolio_mix(500, seed=3)
    S = projection_steps(pol)
    jl = pol["product"] == 1
    want = (3 * S[~jl].sum() + 16 * S[jl].sum()) * 7
    assert bench.algorithmic_flops(pol, 7) == pytest.approx(float(want), rel=0, abs=0)
