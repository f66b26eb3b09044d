"""The benchmark's accounting (no GPU): the algorithmic work per unit it reports against the
constraint and moment counts of the method, and the sources it quotes.

Counts (Sec. II.B): a fluon population carries N_f = 1 + D + D(D+1)/2 + D^2 constraints
(mass, momentum, the second moments, the heat-flux moments c_a^2 c_g of Eq. IIB14-16), a
phonon population N_g = 1 + D + D(D+1)/2 (Eq. IIB16-17); a cell stores n_mom = 1 + D +
D(D+1)/2 + D + 1 + D moments (Eq. IIB5).  Per stencil point and Newton pass the naive
assembly costs 2(2N + N(N+1)/2) FLOP: one multiply-add per constraint for the exponent and
the residual, and one per entry of the packed symmetric Jacobian.
"""
import os

import pytest

import bench
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("D", [1, 2, 3])
def test_counts_match_the_method_and_the_oracle(D):
    nf = 1 + D + D * (D + 1) // 2 + D * D
    ng = 1 + D + D * (D + 1) // 2
    nm = 1 + D + D * (D + 1) // 2 + D + 1 + D
    assert (bench.N_F[D], bench.N_G[D], bench.N_M[D]) == (nf, ng, nm)
    assert (O.nf(D), O.ng(D), O.nmom(D)) == (nf, ng, nm)


def test_per_point_flops_are_the_naive_assembly():
    # 1D / 2D / 3D fluons and phonons
    assert [bench.newton_flops(bench.N_F[D]) for D in (1, 2, 3)] == [36, 150, 456]
    assert [bench.newton_flops(bench.N_G[D]) for D in (1, 2, 3)] == [24, 66, 150]
    for n in range(1, 25):  # brute force: count the multiply-adds one by one
        fma = n + n + sum(1 for a in range(n) for b in range(a, n))
        assert bench.newton_flops(n) == 2 * fma


def test_whole_job_rate():
    # 16,777,216 cells x 10 steps in 1 s -> 167.77 MLUPS; the slowest rank's time divides
    assert bench.whole_job_mlups(4096 * 4096, 10, 1000.0) == pytest.approx(167.77216)
    assert bench.rank_reduce(3.5, "max", 1, None) == 3.5


def test_quoted_traffic_sources_exist():
    assert not set(bench.DRAM_PER_STEP) & set(bench.STALE_DRAM_PER_STEP)
    for table in (bench.DRAM_PER_STEP, bench.STALE_DRAM_PER_STEP):
        for key, (nbytes, src) in table.items():
            assert nbytes > 0
            path = os.path.join(ROOT, src.split(" ")[0])
            assert os.path.exists(path), (key, path)
