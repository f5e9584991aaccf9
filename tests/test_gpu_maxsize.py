"""The largest instance the library accepts (n = 16384): both evaluators
against the oracle on sampled chromosomes, and a short GA solve with the
allocation local search, in one GPU test (the instance takes a few seconds
to generate and ~3 GB of host memory for the oracle's fp64 copies)."""
import numpy as np
import pytest

from gpu_util import need_gpu
from oracle import cost
from paper_1704_06258_gb300 import synth
from paper_1704_06258_gb300.binding import PATH_PLAIN_FP32, PATH_SPLIT_BF16, Instance

pytestmark = pytest.mark.gpu
TOL = {PATH_PLAIN_FP32: 1e-5, PATH_SPLIT_BF16: 1e-4}
N_MAX = 16384


def test_maximum_n_both_paths_and_solve():
    need_gpu()
    inst = synth.large_uniform(seed=1016, n=N_MAX, p=20)
    B = 32
    hubs, S = synth.random_population(1017, inst.n, inst.p, B)
    sample = [0, B - 1]
    ref = np.array([cost.three_term_cost(inst.W, inst.C, inst.chi, inst.alpha, inst.delta, hubs[b], S[b])[0]
                    for b in sample])
    with Instance.from_instance(inst) as gi:
        info = gi.info()
        assert (info["n"], info["ns"], info["tc_folded"]) == (N_MAX, N_MAX, 1)
        for path in (PATH_PLAIN_FP32, PATH_SPLIT_BF16):
            gi.set_params(path=path)
            got = gi.eval(hubs, S)
            assert np.all(np.isfinite(got))
            rel = np.abs(got[sample] - ref) / ref
            assert rel.max() <= TOL[path], (path, rel)
        gi.set_params(islands=2, island_size=32, n1=2, path=PATH_SPLIT_BF16, local_search=1)
        r = gi.solve(3, 19)
    cost.check_allocation(inst.n, r["hubs"], r["S"])
    assert abs(r["cost_fp32"] - r["cost_fp64"]) / r["cost_fp64"] <= TOL[PATH_SPLIT_BF16]
