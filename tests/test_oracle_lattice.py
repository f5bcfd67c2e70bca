"""Pins for the oracle's lattice, Hamiltonian and exact enumeration (§II.A).

The Edwards-Anderson energy and the exact density of states g(k) are checked
against facts fixed by the mathematics rather than by the oracle's own formula:
ferromagnet and Neel ground states, the high-temperature expansion of Z (whose
low-order coefficients are sums over short closed loops, counted here by brute
force over bond subsets), gauge invariance, the spin-flip and sublattice
symmetries, and the beta = 0 energy variance.
"""
import itertools
from math import comb

import numpy as np
import pytest


def bond_list(L):
    """(endpoint a, endpoint b) of bond (n, d) for n = x + L(y + Lz), d = x, y, z."""
    bonds = []
    for z in range(L):
        for y in range(L):
            for x in range(L):
                n = x + L * (y + L * z)
                for d in range(3):
                    c = [x, y, z]
                    c[d] = (c[d] + 1) % L
                    bonds.append((n, c[0] + L * (c[1] + L * c[2])))
    return bonds


def loop_coefficients(L, J, max_len=4):
    """Coefficient of tanh(beta)^m in Z / (2^N cosh^{3N} beta), m <= max_len:
    the sum over even subgraphs (every vertex of even degree) with m bonds of the
    product of their couplings.  Brute force over bond subsets."""
    bonds = bond_list(L)
    masks = [(1 << a) ^ (1 << b) for a, b in bonds]
    nb = len(bonds)
    coeff = [0] * (max_len + 1)
    coeff[0] = 1
    for m in range(1, min(max_len, 3) + 1):
        for sub in itertools.combinations(range(nb), m):
            x = 0
            for i in sub:
                x ^= masks[i]
            if x == 0:
                coeff[m] += int(np.prod([int(J[i]) for i in sub]))
    if max_len >= 4:
        # 4-subsets with zero XOR = pairs of disjoint bond pairs with equal XOR (each counted 3 times)
        groups = {}
        for i, j in itertools.combinations(range(nb), 2):
            groups.setdefault(masks[i] ^ masks[j], []).append((i, j))
        total = 0
        for pairs in groups.values():
            for (a, b), (c, d) in itertools.combinations(pairs, 2):
                if len({a, b, c, d}) == 4:
                    total += int(J[a]) * int(J[b]) * int(J[c]) * int(J[d])
        assert total % 3 == 0
        coeff[4] = total // 3
    return coeff


def expansion_from_levels(L, g, max_len):
    """P(t) = 2^{-N} sum_k g(k) (1-t)^k (1+t)^{3N-k}, exact integer coefficients."""
    N = L ** 3
    nb = 3 * N
    coeff = [0] * (nb + 1)
    for k, gk in enumerate(g):
        gk = int(gk)
        if gk == 0:
            continue
        # (1-t)^k (1+t)^{nb-k}: convolve binomial rows
        a = [comb(k, i) * (-1) ** i for i in range(k + 1)]
        b = [comb(nb - k, i) for i in range(nb - k + 1)]
        for m in range(max_len + 1):
            s = 0
            for i in range(max(0, m - (nb - k)), min(m, k) + 1):
                s += a[i] * b[m - i]
            coeff[m] += gk * s
    out = []
    for m in range(max_len + 1):
        assert coeff[m] % (2 ** N) == 0
        out.append(coeff[m] // 2 ** N)
    return out


@pytest.mark.parametrize("L,seed", [(2, 1), (2, 9), (3, 4), (3, 77)])
def test_enumeration_matches_high_temperature_expansion(oracle_lib, L, seed):
    J = oracle_lib.couplings(L, seed)
    g = oracle_lib.enumerate_levels(L, J)
    assert g.sum() == 2 ** (L ** 3)
    got = expansion_from_levels(L, g, 4)
    want = loop_coefficients(L, J, 4)
    assert got == want


def test_enumeration_ferromagnet_degeneracies(oracle_lib):
    for L in (2, 3):
        N = L ** 3
        J = np.ones(3 * N, dtype=np.int8)
        g = oracle_lib.enumerate_levels(L, J)
        assert g[0] == 2                  # all up, all down
        assert g[1:6].sum() == 0          # the cheapest excitation breaks 6 bonds
        assert g[6] == 2 * N              # single flipped spin (and its mirror)


def test_enumeration_symmetries(oracle_lib):
    rng = np.random.default_rng(5)
    for L in (2, 3):
        N = L ** 3
        J = oracle_lib.couplings(L, 31)
        g = oracle_lib.enumerate_levels(L, J)
        # gauge transformation J'(n,d) = e_n J(n,d) e_{n+d} leaves g unchanged
        e = rng.choice([-1, 1], size=N)
        Jg = np.array([J[3 * n + d] * e[a] * e[b] for n in range(N) for d in range(3)
                       for (a, b) in [bond_list(L)[3 * n + d]]], dtype=np.int8)
        assert np.array_equal(oracle_lib.enumerate_levels(L, Jg), g)
        if L % 2 == 0:
            # bipartite lattice: flipping one sublattice maps E -> -E
            assert np.array_equal(g, g[::-1])
        # beta = 0: <E> = 0 and var E = sum over bond pairs of J_b J_b' <s s s' s'>
        k = np.arange(3 * N + 1)
        E = 2 * k - 3 * N
        mean = (g * E).sum() / 2 ** N
        var = (g * E * E).sum() / 2 ** N - mean ** 2
        bonds = bond_list(L)
        expect = 3 * N
        for i, j in itertools.combinations(range(3 * N), 2):
            if sorted(bonds[i]) == sorted(bonds[j]):      # parallel bonds (L = 2 only)
                expect += 2 * int(J[i]) * int(J[j])
        assert mean == 0
        assert var == pytest.approx(expect, abs=1e-9)


def test_energy_ground_states(oracle_lib):
    for L in (2, 4, 6):
        N = L ** 3
        Jf = np.ones(3 * N, dtype=np.int8)
        up = np.ones(N, dtype=np.int8)
        assert oracle_lib.energy(L, Jf, up) == -3 * N
        assert oracle_lib.energy(L, -Jf, up) == 3 * N
        x, y, z = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
        neel = np.where((x + y + z) % 2 == 0, 1, -1).astype(np.int8).transpose(2, 1, 0).ravel()
        assert oracle_lib.energy(L, Jf, neel) == 3 * N
        assert oracle_lib.energy(L, -Jf, neel) == -3 * N
        one = up.copy()
        one[N // 2 + 1] = -1
        assert oracle_lib.energy(L, Jf, one) == -3 * N + 12
    assert oracle_lib.energy(3, np.ones(81, dtype=np.int8), np.ones(27, dtype=np.int8)) == -81


def test_couplings_balanced_and_seeded(oracle_lib):
    J = oracle_lib.couplings(10, 3)
    assert set(np.unique(J)) == {-1, 1}
    n = J.size
    assert abs((J == 1).mean() - 0.5) < 5 * 0.5 / np.sqrt(n)
    assert np.array_equal(J, oracle_lib.couplings(10, 3))
    assert not np.array_equal(J, oracle_lib.couplings(10, 4))


def test_metropolis_thresholds_limits(oracle_lib):
    thr0 = oracle_lib.metropolis_thresholds(0.0)
    assert list(thr0) == [2 ** 32 - 1] * 3
    for beta in (0.1, 0.7, 2.5):
        thr = oracle_lib.metropolis_thresholds(beta)
        for m in range(3):
            p = np.exp(-4 * (m + 1) * beta)
            assert abs(int(thr[m]) / 2 ** 32 - p) <= 2 ** -32
    assert list(oracle_lib.metropolis_thresholds(50.0)) == [0, 0, 0]
