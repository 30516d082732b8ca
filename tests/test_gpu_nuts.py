"""GPU parity of the NUTS outer move (trajectories built in lockstep, a forward + adjoint pass of
the N filters at every point) against the oracle's NUTS sampler, which runs each sample's
trajectory on its own.  The oracle follows the GPU's decisions only where its own margin is
within the band: a selection or merge whose log-uniform lies within 1e-3 of the log-weight
ratio, a U-turn product within 1e-3 of zero relative to its factors, and, inside the filter
at every trajectory point (the GPU keeps each point's tape), an ancestor decision within the
filters' near-tie band.  Every such tie is counted; every other difference is a mismatch and
must not occur."""
from dataclasses import replace

import numpy as np
import pytest

import oracle.smc2 as osmc2
from paper_2407_17296_gb300 import workloads as W

from .parity import BAND, BAND_REL, TIE_REPORT
from .test_gpu_smc2 import _compare, _stable_lg

pytestmark = pytest.mark.gpu


def _run_gpu_nuts(w, K, **kw):
    from paper_2407_17296_gb300 import binding
    recs, hints = [], []
    P = 2 ** w.nuts_depth - 1
    with binding.Handle(binding.config_for(w, **kw)) as h:
        h.set_point_trace(True)
        for k in range(K):
            st = h.step()
            anc, flag, oanc, ores = h.trace()
            th, lw = h.samples()
            hint = {"outer_anc": oanc, "outer_flag": ores}
            if k == 0:  # iteration 1 runs one filter launch at the prior draws
                hint.update(pf_anc=anc, pf_flag=flag)
            else:       # the move's decisions and the tape of each trajectory point
                tr = h.nuts_trace()
                hint["nuts"] = [{"sel": int(tr["sel"][i]), "merge": int(tr["merge"][i]),
                                 "stop": (int(tr["stop_point"][i]), int(tr["stop_kind"][i]))}
                                for i in range(w.N)]
                # every trajectory point's filter tape, to follow the filters' near-ties there
                hint["nuts_pf"] = [h.point_trace(s) for s in range(P)]
            recs.append(dict(st, theta=th, logw=lw))
            hints.append(hint)
    return recs, hints


def _nuts_counts(ref, hints, stable=None):
    """Decision counts of the oracle's moves; ties and mismatches only for samples whose start
    and selected point are stable (an explosive linear-Gaussian sample, |a| >= 1, separates its
    FP32 and FP64 filters like |a|^t and has negligible weight)."""
    c = {"nuts_ties": 0, "nuts_mismatch": 0, "points": 0, "stop_kinds": [0] * 5, "depths": {},
         "explosive_excluded": 0}
    for prev, r, hint in zip([None] + ref[:-1], ref, hints):
        if "nuts" not in r:
            continue
        th_start = prev["theta"][prev["ancestors"]] if prev["resampled"] else prev["theta"]
        for i, m in enumerate(r["nuts"]):
            if stable is not None and not (stable(th_start[i]) and stable(r["theta"][i])):
                c["explosive_excluded"] += 1
            else:
                c["nuts_ties"] += m["stats"]["nuts_ties"]
                c["nuts_mismatch"] += m["stats"]["nuts_mismatch"]
            c["points"] += m["stats"]["points"]
            c["stop_kinds"][m["stop"][1]] += 1
            c["depths"][m["depth"]] = c["depths"].get(m["depth"], 0) + 1
            # the oracle followed the GPU's decisions: where it stopped is the GPU's stop
            assert tuple(m["stop"]) == hint["nuts"][i]["stop"], (r["k"], i, m["stop"], hint["nuts"][i])
    return c


@pytest.mark.parametrize("weight", [0, 1])
def test_smc2_nuts_matches_oracle(weight):
    """lg1 (N=64, M=128, T=60), 5 iterations, trajectories of up to 7 points, both L-kernels."""
    w = replace(W.lg1(N=64, M=128, T=60, K=5, proposal="nuts"), nuts_depth=3, nuts_weight=weight, gamma=0.1)
    recs, hints = _run_gpu_nuts(w, w.K)
    ref, rec_ref = osmc2.run(w.family, 1, 1, None, w.y, w.N, w.M, w.K, w.gamma, "nuts", w.seed,
                             hints=hints, band=BAND, flag_band=BAND, band_rel=BAND_REL, nuts_depth=3,
                             nuts_unit_weight=(weight == 0))
    name = f"smc2 lg1 nuts depth 3 weight {weight} N=64 M=128 T=60 K=5"
    _compare(recs, ref, rec_ref, stable=_stable_lg(1), name=name, M=w.M)
    c = _nuts_counts(ref, hints, _stable_lg(1))
    TIE_REPORT[name]["nuts"] = c
    print(f"\n[{name}] {c}")
    assert c["nuts_mismatch"] == 0, c
    assert c["nuts_ties"] <= 0.01 * c["points"] + 2, c
    assert c["stop_kinds"][1] + c["stop_kinds"][3] > 0  # the trajectories do turn


def test_nuts_sv_matches_oracle():
    """SV (N=32, M=128, T=60), 4 iterations, depth 2: another model family through the move."""
    w = replace(W.sv(T=60, N=32, M=128, K=4, proposal="nuts"), nuts_depth=2)
    recs, hints = _run_gpu_nuts(w, w.K)
    ref, rec_ref = osmc2.run(w.family, 1, 1, None, w.y, w.N, w.M, w.K, w.gamma, "nuts", w.seed,
                             hints=hints, band=BAND, flag_band=BAND, band_rel=BAND_REL, nuts_depth=2)
    name = "smc2 sv nuts depth 2 N=32 M=128 T=60 K=4"
    _compare(recs, ref, rec_ref, name=name, M=w.M)
    c = _nuts_counts(ref, hints)
    TIE_REPORT[name]["nuts"] = c
    assert c["nuts_mismatch"] == 0, c


def test_nuts_trace_and_launches():
    """The trace is readable after a NUTS move only; every sample stops with a valid kind at a
    point inside its trajectory; an iteration launches begin + 7 x (filters + point) + finish +
    the update."""
    from paper_2407_17296_gb300 import binding
    w = replace(W.lg1(N=64, M=128, T=40, K=3, proposal="nuts"), nuts_depth=3)
    with binding.Handle(binding.config_for(w)) as h:
        h.step()
        with pytest.raises(binding.Smc2Error):
            h.nuts_trace()  # iteration 1 draws from the prior: no move yet
        before = binding.kernel_launches()
        h.step()
        after = binding.kernel_launches()
        tr = h.nuts_trace()
    assert np.all((tr["stop_kind"] >= 0) & (tr["stop_kind"] <= 4))
    moved = tr["stop_kind"] != 4
    assert np.all((tr["stop_point"][moved] >= 0) & (tr["stop_point"][moved] <= 6))
    # point s = 2^j - 1 + n is selected only if it was built (s <= stop point)
    for i in np.nonzero(moved)[0]:
        assert int(tr["sel"][i]) >> (int(tr["stop_point"][i]) + 1) == 0
    assert after - before > 7  # the launch counter saw the trajectory's points
