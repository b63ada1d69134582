"""Host-side checks of the solver's memory-planning rules (csrc/plan_rules.h), compiled with the
host C++ compiler: the batched plan's restart length against kept factors, and the number of
systems whose factors a refinement keeps when not all fit."""
import os
import shutil
import subprocess

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2504_07269_gb300", "csrc")
GiB = 1 << 30

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include "plan_rules.h"
int main(int argc, char** argv) {
    if (argv[1][0] == 'r') {   // r N avail factors m m_min
        std::printf("%d\n", stfdm::batch_restart_for_factors(std::strtoull(argv[2], 0, 10), std::strtoull(argv[3], 0, 10),
                                                            std::strtoull(argv[4], 0, 10), std::atoi(argv[5]), std::atoi(argv[6])));
    } else if (argv[1][0] == 's') {   // s N n_t grid per avail fixed m m_min
        std::printf("%d\n", stfdm::single_restart_for_partial_keep(
            std::strtoull(argv[2], 0, 10), std::atoi(argv[3]), std::atoi(argv[4]), std::strtoull(argv[5], 0, 10),
            std::strtoull(argv[6], 0, 10), std::strtoull(argv[7], 0, 10), std::atoi(argv[8]), std::atoi(argv[9])));
    } else {                   // k n_t grid per avail fixed
        std::printf("%d\n", stfdm::partial_keep_systems(std::atoi(argv[2]), std::atoi(argv[3]), std::strtoull(argv[4], 0, 10),
                                                       std::strtoull(argv[5], 0, 10), std::strtoull(argv[6], 0, 10)));
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def rules(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("rules")
    src, exe = d / "drv.cpp", d / "drv"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", HDR, str(src), "-o", str(exe)], check=True)

    def call(*args):
        return int(subprocess.run([str(exe)] + [str(a) for a in args], check=True, capture_output=True,
                                  text=True).stdout)
    return call


def basis(N, m):
    return N * ((m + 1) * 16 + m * 8)


def room(avail):
    return int((avail - 2 * GiB) * 0.9) if avail > 2 * GiB else 0


@pytest.mark.parametrize("N,avail,factors", [
    (10_000_000, 200 * GiB, 10 * GiB),      # everything fits: the longest basis
    (370_366_154, 240 * GiB, 415 * 10**9),  # the 64-problem batch: factors far beyond memory
    (100_000_000, 200 * GiB, 120 * GiB),    # in between
    (100_000_000, 3 * GiB, 0),              # tiny memory: the half-memory cap alone
    (1_000, 1 * GiB, 0),
])
def test_batch_restart_yields_to_kept_factors(rules, N, avail, factors):
    m0, m_min = 20, 4
    m = rules("r", N, avail, factors, m0, m_min)
    assert 2 <= m <= m0
    # never more than half the memory for the basis (unless already at the floor of 2)
    assert m == 2 or basis(N, m) <= avail // 2
    # the basis leaves room for every keepable factor, unless it is at its shortest
    assert m <= m_min or basis(N, m) + factors <= room(avail)
    # and it is the longest such basis
    if m < m0:
        assert basis(N, m + 1) > avail // 2 or (m + 1 > m_min and basis(N, m + 1) + factors > room(avail))


def test_batch_restart_at_the_64_problem_batch(rules):
    probs = synth.batch_problems(64, 5)
    N = sum(pr.n_t * pr.n_x for pr in probs)
    factors = sum((pr.n_t * pr.n_x * (pr.n + 1) * 8 + 255) // 256 * 256 for pr in probs)   # b = n
    assert N == 370_366_154
    assert rules("r", N, 250 * GiB, factors, 20, 4) == 4
    assert rules("r", N, 250 * GiB, 0, 20, 4) > 4            # without kept factors the basis stays long


@pytest.mark.parametrize("avail_gb", [75, 120, 180, 240, 400, 10_000])
def test_partial_keep_fills_whole_waves(rules, avail_gb):
    # 384^2 squares, P2 time n_t = 1024: b = 384, one CTA per SM on 152 SMs
    n_t, grid, n_x, b = 1024, 152, 383 * 383, 384
    per = n_x * (b + 1) * 8
    fixed = grid * per + grid * (b + 32) * (b + 1) * 8 + 2 * GiB
    avail = avail_gb * 10**9
    K = rules("k", n_t, grid, per, avail, fixed)
    kmax = int((avail - fixed) * 0.9 / per) if avail > fixed else 0
    if kmax <= 0 or kmax >= n_t:
        assert K == 0                           # none fit, or all do (then everything is kept)
        return
    assert 0 <= K <= kmax                       # fits
    assert (n_t - K) % grid == 0 or K == 0      # the refactorised systems fill whole waves
    assert K == 0 or K > kmax - grid            # no whole wave left unused


@pytest.mark.parametrize("avail_gb", [150, 200, 260, 290, 400])
def test_single_restart_drops_refactorisation_waves(rules, avail_gb):
    """384^2 squares, P2 time n_t = 1024 (150M unknowns, 463 GB of factors): the restart length is
    the longest that needs no more refactorisation waves than the shortest basis."""
    n_t, grid, n_x, b = 1024, 152, 383 * 383, 384
    N = n_t * n_x
    per = n_x * (b + 1) * 8
    fixed = grid * per + grid * (b + 32) * (b + 1) * 8 + 2 * GiB
    avail = avail_gb * 10**9
    m0, m_min = 20, 4
    m = rules("s", N, n_t, grid, per, avail, fixed, m0, m_min)

    def waves(mm):
        bb = N * (2 * mm + 1) * 16
        K = rules("k", n_t, grid, per, avail - bb, fixed) if bb < avail else 0
        return (n_t - K + grid - 1) // grid

    cap = m0
    while cap > 2 and N * (2 * cap + 1) * 16 > avail // 3:
        cap -= 1
    lo = min(m_min, cap)
    assert lo <= m <= cap
    assert waves(m) == waves(lo)                    # no wave more than the shortest basis needs
    assert m == cap or waves(m + 1) > waves(lo)      # and the longest such basis
    if avail_gb == 290:
        assert waves(m) < waves(cap)                # at the full memory the long basis costs a wave
