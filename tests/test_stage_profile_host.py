"""The stage-clock summary of stage_profile (host arithmetic, no GPU)."""
import numpy as np

from paper_2411_14754_gb300 import stage_profile as SP


def test_summary_of_synthetic_stamps():
    # 3 queries, clusters of 2: CTA r of query q stamps slot s at 1000 q + 10 s + r,
    # so every stage lasts 10 cycles; CTA 0 stamps the merge 7 cycles after
    # slot 15; slots 18 and 19 hold the S4 split; unused CTA rows are -1
    nq, CL = 3, 2
    clk = np.full((nq, 16, 20), -1, np.int64)
    for q in range(nq):
        for r in range(CL):
            clk[q, r, 0] = r
            for s in range(1, 16):
                clk[q, r, s] = 1000 * q + 10 * s + r
            clk[q, r, 18], clk[q, r, 19] = 4, 5
        clk[q, 0, 16] = clk[q, 0, 15] + 7
    res = SP.summarise(clk)
    assert res["cluster_size"] == CL and res["queries"] == nq
    assert res["mean_query_cycles"] == 140.0
    per = {r["stage"]: r for r in res["stages"]}
    for name, a, b in SP.STAGES:
        assert per[name]["cycles"] == 10.0 * (b - a)
    assert abs(sum(r["share"] for r in res["stages"][:-1]) - 1.0) < 1e-12
    assert per["merge of the local top-k lists (CTA 0)"]["cycles"] == 7.0
    assert res["s4_split"] == {"list_segments": 4.0, "scan": 5.0}
