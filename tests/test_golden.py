"""The stored fixture tests/golden/bc_small.txt (exact rational BC of small graphs, Eq. 1)
against what fixes it independently of the oracle that wrote it: closed forms of Eq. 1 for
its families, the invariant sum_v BC(v) = sum over ordered connected pairs of (d - 1), and
a rerun of its generator; the C oracle must agree with it, with and without the 1-degree
reduction."""
import os
import sys
from fractions import Fraction

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import brute

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_golden  # noqa: E402

FIX = {name: (n, edges, bc) for name, n, edges, bc in make_golden.load()}


def test_fixture_is_what_the_generator_writes():
    assert open(make_golden.FIXTURE).read() == make_golden.render()


def test_closed_forms():
    """Ordered pairs (twice the unordered closed forms)."""
    n, _, bc = FIX["path7"]
    assert bc == [2 * i * (n - 1 - i) for i in range(n)]
    n, _, bc = FIX["star6"]
    assert bc == [(n - 1) * (n - 2)] + [0] * (n - 1)
    k = 3  # C_{2k+1}: each vertex k(k-1)/2 unordered
    assert FIX["cycle7"][2] == [k * (k - 1)] * 7
    k = 4  # C_{2k}: each vertex (k-1)^2/2 unordered
    assert FIX["cycle8"][2] == [(k - 1) ** 2] * 8
    a, b = 3, 4  # K_{a,b}: side a gets C(b,2)/a unordered, side b gets C(a,2)/b
    assert FIX["k3_4"][2] == [Fraction(b * (b - 1), a)] * a + [Fraction(a * (a - 1), b)] * b
    # Petersen: distance 2 pairs (30 unordered) each have one middle vertex; vertex-transitive
    assert FIX["petersen"][2] == [6] * 10
    # bowtie: the 2 x 2 pairs across the shared vertex pass through it, nothing else
    assert FIX["bowtie"][2] == [0, 0, 8, 0, 0]


@pytest.mark.parametrize("name", sorted(FIX))
def test_sum_invariant(name):
    n, edges, bc = FIX[name]
    g = gg.from_edge_list(n, edges)
    assert sum(bc) == brute.ordered_pair_distance_sum(g)


@pytest.mark.parametrize("name", sorted(FIX))
def test_c_oracle_agrees(name):
    n, edges, bc = FIX[name]
    g = gg.from_edge_list(n, edges)
    want = np.array([float(x) for x in bc])
    for prune in (False, True):
        got = oracle.bc_exact(g, prune=prune)
        assert np.all(np.abs(got - want) <= 1e-12 * np.maximum(np.abs(want), 1.0)), (name, prune)
