"""The float64 vertex coordinates: the library's integer-quotient conversion
against exact rationals at the extremes of its domain.

A vertex of a cell is p + N / D with exact integers (the meeting point of
two lines, Section 3; Section 5 stores the vertices).  The compaction kernel
writes each coordinate as the quotient num / D of integers with
0 <= num < 2^63 and 0 < D < 2^44 by a float-float division (Dekker 1971),
with a stated error of at most 2^-42 q + 2^-39 for the exact quotient q and
exact integer quotients.  vor_vertex_quotients runs that same device code.
"""

from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1212_1095_gb300 as vg  # noqa: E402


def _cases():
    rng = np.random.default_rng(2024)
    nums, dens = [], []

    def add(a, d):
        if 0 <= a < (1 << 63) and 0 < d < (1 << 44) and a // d < (1 << 21):
            nums.append(int(a))
            dens.append(int(d))

    # denominators near 2^43 and numerators near 2^63 (q near 2^20)
    for d in [(1 << 43) - 1, (1 << 43) - 12345, (1 << 43) + 7, (1 << 42) + 1, 3 << 41]:
        for q in [(1 << 20), (1 << 20) - 1, 1, 0, 524287]:
            add(q * d, d)                                   # integer quotients
            add(q * d + 1, d)
            add(q * d + d // 2, d)
            add(max(q * d - 1, 0), d)
        add((1 << 63) - 1, d)
    # random magnitudes over the whole domain
    for _ in range(20000):
        d = int(rng.integers(1, 1 << int(rng.integers(1, 44))))
        qmax = min((1 << 21) - 1, ((1 << 63) - 1) // d)
        q = int(rng.integers(0, qmax + 1))
        r = int(rng.integers(0, d))
        add(q * d + r, d)
        add(q * d, d)
    # small denominators, fractions near integers and near zero
    for d in [1, 2, 3, 7, 1 << 20, (1 << 21) + 1]:
        for a in [0, 1, d - 1, d, d + 1, 5 * d + 1, ((1 << 20) * d) - 1]:
            add(a, d)
    return nums, dens


def test_vertex_quotients_error_bound_at_the_extremes():
    nums, dens = _cases()
    num = torch.tensor(nums, dtype=torch.int64, device="cuda")
    den = torch.tensor([d if d < (1 << 63) else d - (1 << 64) for d in dens], dtype=torch.int64,
                       device="cuda")
    got = vg.vor_vertex_quotients(num, den).cpu().numpy()
    worst = 0.0
    for a, d, g in zip(nums, dens, got):
        q = Fraction(a, d)
        err = abs(Fraction(float(g)) - q)
        bound = Fraction(1, 1 << 42) * q + Fraction(1, 1 << 39)
        assert err <= bound, (a, d, float(g), float(q))
        if q.denominator == 1:
            assert Fraction(float(g)) == q, ("integer quotient not exact", a, d, float(g))
        worst = max(worst, float(err / bound))
    print(f"{len(nums)} quotients, worst error {worst:.3f} of the bound")


def test_vertex_quotients_reject_outside_the_domain():
    num = torch.tensor([-1, 5, 1 << 62, 7], dtype=torch.int64, device="cuda")
    den = torch.tensor([3, 0, 1, 1 << 44], dtype=torch.int64, device="cuda")
    got = vg.vor_vertex_quotients(num, den).cpu().numpy()
    assert np.all(np.isnan(got))
