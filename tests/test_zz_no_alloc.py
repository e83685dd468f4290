"""GPU test of rsv_reserves_noalloc, the valuation entry point for callers that
cannot allocate device memory -- a service whose device memory belongs to a
fixed arena or pool that must stay its only owner, or latency-bound code that
cannot take the implicit synchronisation of cudaMalloc.  Every buffer here is
owned by the caller (torch tensors), and the results must match those of
rsv_compute_reserves on the same inputs, on two calls in a row (the second call
finds the first call's contents in the shared scratch array).

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1401_1757_gb300 import rsv

pytestmark = pytest.mark.gpu

TOL = 1e-6   # the compensated FP32 form's tolerance in the parity tests


def test_noalloc_matches_main_entry_point_on_two_calls():
    tab = synth.gm_monthly_survival()
    pol = synth.portfolio_mix(3000, seed=31)       # all four products, decrement table 0
    v = synth.vasicek_paths(300, 1200, seed=31)
    n, S = 3000, 300

    ctx = rsv.rsv_create(0, torch.cuda.current_stream())
    try:
        rsv.rsv_load_decrements(ctx, 0, tab)
        rsv.rsv_load_portfolio(ctx, pol)
        rsv.rsv_load_scenarios(ctx, v)
        want = np.zeros((n, S))
        want_tot = np.zeros(S)
        rsv.rsv_compute_reserves(ctx, rsv.RSV_FORM_F32_COMP, rsv.RSV_OUT_V0 | rsv.RSV_OUT_SCEN_TOTAL,
                                 V0d=want, scen_total=want_tot)
    finally:
        rsv.rsv_destroy(ctx)

    recs = rsv.policy_records(pol)
    d_pols = torch.from_numpy(recs.view(np.uint8).copy()).cuda()
    d_tab = torch.from_numpy(tab).cuda()
    d_v = torch.from_numpy(np.ascontiguousarray(v.T)).cuda()        # [n_steps][n_scen]
    stream = torch.cuda.current_stream()
    for call in range(2):
        V0 = torch.full((n, S), float("nan"), dtype=torch.float64, device="cuda")
        tot = torch.full((S,), float("nan"), dtype=torch.float64, device="cuda")
        rsv.rsv_reserves_noalloc(0, stream, d_pols, d_tab, d_v, V0, tot)
        got, got_tot = V0.cpu().numpy(), tot.cpu().numpy()
        scale = np.maximum(np.abs(want), 1e-9 * pol["amount"][:, None])
        err = float(np.max(np.abs(got - want) / scale))
        terr = float(np.max(np.abs(got_tot - want_tot) / np.abs(want_tot)))
        print(f"call {call}: max rel diff to rsv_compute_reserves {err:.3e}, totals {terr:.3e}")
        assert err <= TOL and terr <= TOL
        # and against the FP64 oracle directly, on a sample of the policies
        idx = np.arange(0, n, 29)
        ref, _ = oracle.reserves_batch(synth.take(pol, idx), tab, v)
        oerr = float(np.max(np.abs(got[idx] - ref) / np.maximum(np.abs(ref), 1e-9 * pol["amount"][idx, None])))
        print(f"call {call}: max rel err against the oracle {oerr:.3e}")
        assert oerr <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_records():
    lib = rsv.load_library()
    d_tab = torch.from_numpy(synth.gm_monthly_survival()).cuda()
    d_v = torch.ones((1200, 1000), dtype=torch.float64, device="cuda")
    V0 = torch.empty(8, dtype=torch.float64, device="cuda")
    d_pols = torch.zeros(48, dtype=torch.uint8, device="cuda")
    # 10 million policies x 1,000 scenarios: beyond the fixed scratch, refused before any GPU work
    st = lib.rsv_reserves_noalloc(0, None, C.c_void_p(d_pols.data_ptr()), 10_000_000, C.c_void_p(d_tab.data_ptr()),
                                  1440, C.c_void_p(d_v.data_ptr()), 1000, 1200, C.c_void_p(V0.data_ptr()), None)
    assert st == rsv.RSV_E_LIMIT
    # a record naming decrement table 1 (only table 0 exists here)
    pol = synth.portfolio_single_life(1)
    pol["table1"][:] = 1
    bad = torch.from_numpy(rsv.policy_records(pol).view(np.uint8).copy()).cuda()
    out = torch.empty((1, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_reserves_noalloc(0, torch.cuda.current_stream(), bad, d_tab, d_v[:, :4].contiguous(), out)
    assert e.value.status == rsv.RSV_E_ARG
    # the assumptions of Section 3.7 give the status rsv_compute_reserves gives:
    # an amount not finite, a reversion outside [0, 1]; with two bad records,
    # the first one's
    out2 = torch.empty((2, 4), dtype=torch.float64, device="cuda")
    mix = synth.portfolio_mix(2, seed=1)
    mix["product"][:] = [0, 1]
    mix["age2_m"][1], mix["reversion"][1] = 700, 0.6
    for change, want in ((("amount", 0, np.inf), rsv.RSV_E_ASSUMPTION), (("reversion", 1, 1.5), rsv.RSV_E_ASSUMPTION),
                         (("table1", 0, 3), rsv.RSV_E_ARG)):
        p2 = {k: a.copy() for k, a in mix.items()}
        p2[change[0]][change[1]] = change[2]
        if change[0] == "table1":
            p2["amount"][1] = np.nan        # a later record with an assumption broken: the first decides
        d2 = torch.from_numpy(rsv.policy_records(p2).view(np.uint8).copy()).cuda()
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_reserves_noalloc(0, torch.cuda.current_stream(), d2, d_tab, d_v[:, :4].contiguous(), out2)
        assert e.value.status == want, change
