"""Parity of the QAOA landscape workload (Sec. 5.7) on the path its grid search
takes: grid points run as one batch (one captured CUDA graph), in tree mode
(DCP) and in plain baseline mode, FP64 counts bit-exact against the oracle for
the same seeds; and the FP32 landscape estimate of a grid point within sampling
error of the oracle's."""
import numpy as np
import pytest

import paper_2203_13892_gb300 as tqs
from paper_2203_13892_gb300 import qaoa
from tqs_inputs import qaoa_maxcut

pytestmark = pytest.mark.gpu

SHOTS = 512
POINTS = [(5, 7), (20, 3)]  # (gamma index, beta index) on the 31 x 31 grid


def _circuits():
    E = qaoa.graph()
    gammas, betas = qaoa.angles(31)
    return E, [qaoa_maxcut(qaoa.N, E, gammas[i], betas[j]) for i, j in POINTS]


@pytest.mark.parametrize("mode", ["tree", "baseline"])
def test_qaoa_batch_fp64_bit_exact(orc, mode):
    E, circs = _circuits()
    handles = [tqs.circuit(c) for c in circs]
    noises = [tqs.tqs_noise_model(*qaoa.NOISE) for _ in circs]
    b = tqs.tqs_batch_create(handles, noises, [SHOTS] * len(circs), tqs.options(mode=mode, prec="fp64"))
    seeds = [11, 12]
    tqs.tqs_batch_execute(b, seeds)
    for k, c in enumerate(circs):
        got = tqs.tqs_batch_counts(b, k, qaoa.N)
        arity, split = tqs.tqs_partition(handles[k], noises[k], SHOTS, tqs.options(mode=mode))
        want = orc.core.run_tree(c, *qaoa.NOISE, SHOTS, seeds[k], arity, split)
        assert int(got.sum()) == SHOTS
        assert np.array_equal(got, want), (mode, k)
    b.close()


def test_qaoa_fp32_landscape_point_within_sampling_error(orc):
    """The cut fraction the FP32 grid search reads from one histogram agrees with
    the oracle's FP64 tree run of the same seed within 4 standard errors of a
    2,048-shot estimate (the two differ only where FP32 rounding moves a sample
    across an outcome boundary)."""
    E, circs = _circuits()
    cut = qaoa.cut_values(E) / len(E)
    c = circs[0]
    gammas, betas = qaoa.angles(31)
    hist, ms, _ = qaoa.row_histograms(E, gammas[POINTS[0][0]], [betas[POINTS[0][1]]], 2048, [3], "tree", "fp32")
    h, nz = tqs.circuit(c), tqs.tqs_noise_model(*qaoa.NOISE)
    arity, split = tqs.tqs_partition(h, nz, 2048, tqs.options())
    want = orc.core.run_tree(c, *qaoa.NOISE, 2048, 3, arity, split).astype(np.float64) / 2048
    got = hist[0].astype(np.float64) / 2048
    m_want = float(want @ cut)
    se = np.sqrt(max(float(want @ cut ** 2) - m_want ** 2, 1e-12) / 2048)
    assert abs(float(got @ cut) - m_want) < 4 * se
    assert ms > 0
