"""The half-index arithmetic of the slab-resident staples, checked exhaustively on the CPU.

Inside a CTA of the slab-resident kernel the sites of one time slice are numbered
li = x + L (y + L zl) (zl < nz planes) and stored by parity at half index li >> 1.  A
staple of the link (x, mu) reads the links at x + mu, x + nu, x - nu and x + mu - nu
(Section 2.1: the staple of the Wilson action).  The kernel forms each neighbour's half
index as h + (offset formed once per site) and decides whether a z step leaves the CTA from
the site's plane alone.  This module restates both rules and compares them, for every site
and every (mu, nu), with the plain definition (li + s) >> 1 and the bounds test li + s >= P
/ li + s < 0 of the local index."""
from __future__ import annotations

import itertools

import pytest


def steps(x, y, L):
    """Local-index steps (+1 / -1) of the site in x, y (periodic) and z (L^2, not wrapped)."""
    xu = -(L - 1) if x == L - 1 else 1
    xd = L - 1 if x == 0 else -1
    yu = -(L - 1) * L if y == L - 1 else L
    yd = (L - 1) * L if y == 0 else -L
    return {"up": {0: 0, 1: xu, 2: yu, 3: L * L}, "dn": {0: 0, 1: xd, 2: yd, 3: -L * L}}


def half_steps(x, y, L):
    """The kernel's half-index offsets: (b + s) >> 1 with b = x & 1, formed once per site."""
    b = x & 1
    xu = ((b - (L - 1)) >> 1) if x == L - 1 else ((b + 1) >> 1)
    xd = ((b + L - 1) >> 1) if x == 0 else ((b - 1) >> 1)
    yu = -(L - 1) * L // 2 if y == L - 1 else L // 2
    yd = (L - 1) * L // 2 if y == 0 else -L // 2
    zs = L * L // 2
    return {"up": {0: 0, 1: xu, 2: yu, 3: zs}, "dn": {0: 0, 1: xd, 2: yd, 3: -zs}}


@pytest.mark.parametrize("L,nz", [(4, 1), (4, 2), (4, 4), (6, 3), (8, 2), (10, 5), (12, 3), (24, 3)])
def test_half_index_and_edge_rules(L, nz):
    P = L * L * nz
    for zl, y, x in itertools.product(range(nz), range(L), range(L)):
        li = x + L * (y + L * zl)
        h = li >> 1
        st, hs = steps(x, y, L), half_steps(x, y, L)
        zup, zdn = zl == nz - 1, zl == 0
        for mu, nu in itertools.permutations(range(4), 2):
            cases = {
                "mu": (st["up"][mu], hs["up"][mu], 1 if mu == 3 else 0),
                "nu": (st["up"][nu], hs["up"][nu], 1 if nu == 3 else 0),
                "nd": (st["dn"][nu], hs["dn"][nu], -1 if nu == 3 else 0),
                "dg": (st["up"][mu] + st["dn"][nu], hs["up"][mu] + hs["dn"][nu],
                       (1 if mu == 3 else 0) - (1 if nu == 3 else 0)),
            }
            for name, (s, dh, zs) in cases.items():
                li2 = li + s
                assert (li2 >> 1) == h + dh, (L, nz, x, y, zl, mu, nu, name)
                if zs > 0:
                    assert (li2 >= P) == zup, (L, nz, x, y, zl, mu, nu, name)
                    if zup:   # the neighbour CTA's half index
                        assert (li2 - P) >> 1 == h + dh - P // 2
                elif zs < 0:
                    assert (li2 < 0) == zdn, (L, nz, x, y, zl, mu, nu, name)
                    if zdn:
                        assert (li2 + P) >> 1 == h + dh + P // 2
                else:
                    assert 0 <= li2 < P


def test_a_wrong_x_offset_is_caught():
    """Dropping the parity bit from the x offsets (a plausible slip) breaks the identity."""
    L, nz = 6, 2
    bad = 0
    for zl, y, x in itertools.product(range(nz), range(L), range(L)):
        li = x + L * (y + L * zl)
        wrong_xu = (-(L - 1)) // 2 if x == L - 1 else 0   # (s >> 1) instead of ((b + s) >> 1)
        bad += ((li + steps(x, y, L)["up"][1]) >> 1) != (li >> 1) + wrong_xu
    assert bad > 0
