"""The closed forms behind the GPU's EG2 and EG1 arc sums, checked against
quadrature on the CPU (no GPU, no oracle): the moments J_mn = int cos^m sin^n
over the two half-circles that the grid lines through a node cut off, over
their intersection, and over the whole circle; and the inclusion-exclusion
identity that turns the sum over the four cells' arcs (eq. (EG2), a vertex
node) into one whole-circle term and three difference terms.

Frame (reflected so that u', v' >= 0): X = {cos > a} = (-acos a, acos a),
Y = {sin > b} = (asin b, pi - asin b), and X and Y meet in (asin b, acos a)
when a^2 + b^2 < 1.  The formulas below are restated from the calculus
(the recurrences (m + n) J_mn = [cos^(m-1) sin^(n+1)] + (m - 1) J_(m-2)n and
(m + n) J_mn = -[cos^(m+1) sin^(n-1)] + (n - 1) J_m(n-2)), not taken from the
kernel source."""
import numpy as np
import pytest
from scipy.integrate import quad

# (quad reports round-off when a requested tolerance is below what double
# precision reaches on a near-zero integral; the assertions check the values)
pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")

# the (m, n) the EG2 moments use: m, n <= 4, m + n <= 6
PAIRS = [(m, n) for m in range(5) for n in range(5) if m + n <= 6]


def quad_moment(m, n, t0, t1):
    if t1 <= t0:
        return 0.0
    return quad(lambda t: np.cos(t) ** m * np.sin(t) ** n, t0, t1, epsabs=1e-14, epsrel=1e-13, limit=200)[0]


def arc_table(t0, t1):
    """J[m][n] over (t0, t1) from the end points by the two recurrences."""
    c0, s0, c1, s1 = np.cos(t0), np.sin(t0), np.cos(t1), np.sin(t1)
    J = np.zeros((7, 7))

    def br(p, q):  # [cos^p sin^q] from t0 to t1
        return c1 ** p * s1 ** q - c0 ** p * s0 ** q

    J[0][0] = t1 - t0
    J[1][0] = br(0, 1)
    J[0][1] = -br(1, 0)
    for tot in range(2, 7):
        for m in range(tot + 1):
            n = tot - m
            if m >= 2:
                J[m][n] = (br(m - 1, n + 1) + (m - 1) * J[m - 2][n]) / tot
            elif n >= 2:
                J[m][n] = (-br(m + 1, n - 1) + (n - 1) * J[m][n - 2]) / tot
            else:  # m = n = 1
                J[1][1] = 0.5 * br(0, 2)
    return J


def half_table(a):
    """int over (-acos a, acos a) of cos^m sin^n: twice the integral from 0
    for even n, zero for odd n."""
    al = np.arccos(a)
    return arc_table(-al, al)


def full_circle(m, n):
    if m % 2 or n % 2:
        return 0.0
    # 2 pi (m-1)!! (n-1)!! / (m + n)!!
    def dfact(k):
        return 1.0 if k <= 0 else k * dfact(k - 2)
    return 2.0 * np.pi * dfact(m - 1) * dfact(n - 1) / dfact(m + n)


@pytest.mark.parametrize("a", [0.0, 0.17, 0.5, 0.83, 0.999, 1.0])
def test_half_circle_table_matches_quadrature(a):
    al = np.arccos(a)
    H = half_table(a)
    for m, n in PAIRS:
        ref = quad_moment(m, n, -al, al)
        assert abs(H[m][n] - ref) < 1e-13, (a, m, n, H[m][n], ref)
        if n % 2:
            assert abs(H[m][n]) < 1e-14  # symmetric about theta = 0


@pytest.mark.parametrize("b", [0.0, 0.3, 0.71, 1.0])
def test_y_side_is_the_transposed_x_table(b):
    """int over Y = (asin b, pi - asin b) of cos^m sin^n = H_b[n][m]
    (theta -> pi/2 - theta exchanges cos and sin and maps Y onto X)."""
    H = half_table(b)
    for m, n in PAIRS:
        ref = quad_moment(m, n, np.arcsin(b), np.pi - np.arcsin(b))
        assert abs(H[n][m] - ref) < 1e-13, (b, m, n)


def test_whole_circle_and_quarter_arc_match_quadrature():
    for m, n in PAIRS:
        assert abs(full_circle(m, n) - quad_moment(m, n, 0.0, 2.0 * np.pi)) < 1e-12
    rng = np.random.default_rng(11)
    for _ in range(12):
        a, b = rng.uniform(0.0, 0.7, 2)
        J = arc_table(np.arcsin(b), np.arccos(a))
        for m, n in PAIRS:
            assert abs(J[m][n] - quad_moment(m, n, np.arcsin(b), np.arccos(a))) < 1e-13


def _weights():
    # the EG2 weights: 1, cos, sin, cos^2 - 1/4, sin cos, sin^2 - 1/4 (as monomial pairs)
    return [{(0, 0): 1.0}, {(1, 0): 1.0}, {(0, 1): 1.0}, {(2, 0): 1.0, (0, 0): -0.25}, {(1, 1): 1.0},
            {(0, 2): 1.0, (0, 0): -0.25}]


def _moment(coef, w, table):
    """int of (sum_ie coef[i][e] cos^i sin^e) * w against a moment table."""
    return sum(coef[i][e] * wv * table(i + dm, e + dn) for i in range(3) for e in range(3) for (dm, dn), wv in w.items())


@pytest.mark.parametrize("seed", range(6))
def test_inclusion_exclusion_equals_the_sum_over_the_four_arcs(seed):
    """Per-cell polynomials b_q (degree <= 2 in each of cos and sin) on the
    four quadrant arcs of a vertex circle: the direct sum of the arc
    integrals equals circle(b_--) + X(b_+- - b_--) + Y(b_-+ - b_--) +
    (X and Y)(b_++ - b_+- - b_-+ + b_--), for lines that cross the circle
    and for lines that miss it."""
    rng = np.random.default_rng(seed)
    a, b = (rng.uniform(0.0, 0.65, 2) if seed % 2 == 0 else rng.uniform(0.0, 1.0, 2))
    a, b = min(a, 1.0), min(b, 1.0)
    B = {q: rng.normal(size=(3, 3)) for q in ("++", "+-", "-+", "--")}
    alx, aly = np.arccos(a), np.arcsin(b)
    meet = a * a + b * b < 1.0
    # quadrant arcs: ++ = X and Y, +- = X not Y, -+ = Y not X, -- = neither
    # (X = (-alx, alx), Y = (aly, pi - aly), both within (-pi/2, 3 pi/2); when
    # the lines miss each other inside the circle, the gap (alx, aly) between
    # X and Y is the -- cell's too)
    arcs = {"++": [(aly, alx)] if meet else [],
            "+-": [(-alx, min(aly, alx))],
            "-+": [(max(aly, alx), np.pi - aly)],
            "--": [(np.pi - aly, 2.0 * np.pi - alx)] + ([] if meet else [(alx, aly)])}
    Hx, Hy = half_table(a), half_table(b)
    Jq = arc_table(aly, alx) if meet else np.zeros((7, 7))
    for w in _weights():
        direct = 0.0
        for q, coef in B.items():
            def f(t, coef=coef):
                c, sn = np.cos(t), np.sin(t)
                poly = sum(coef[i][e] * c ** i * sn ** e for i in range(3) for e in range(3))
                return poly * sum(wv * c ** dm * sn ** dn for (dm, dn), wv in w.items())
            for t0, t1 in arcs[q]:
                if t1 > t0:
                    direct += quad(f, t0, t1, epsabs=1e-13, epsrel=1e-13, limit=200)[0]
        ie = (_moment(B["--"], w, full_circle) + _moment(B["+-"] - B["--"], w, lambda m, n: Hx[m][n])
              + _moment(B["-+"] - B["--"], w, lambda m, n: Hy[n][m])
              + _moment(B["++"] - B["+-"] - B["-+"] + B["--"], w, lambda m, n: Jq[m][n]))
        assert abs(ie - direct) < 1e-11 * (1.0 + abs(direct)), (seed, w, ie, direct)


@pytest.mark.parametrize("a,b", [(0.2, 0.3), (0.6, 0.7), (0.9, 0.1), (1.0, 0.4), (0.0, 0.0)])
def test_eg1_closed_forms(a, b):
    """EG1 on piecewise-constant data needs (1, cos, sin, cos^2, cos sin,
    sin^2) over X, Y and X and Y: X gives (2 al, 2 s, 0, al + a s, 0,
    al - a s) with al = acos a, s = sin al; Y the same with cos and sin
    exchanged; X and Y from its end points (sin aly, b) and (a, sin alx)."""
    al, s = np.arccos(a), np.sqrt(max(0.0, 1.0 - a * a))
    X = [2 * al, 2 * s, 0.0, al + a * s, 0.0, al - a * s]
    mons = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    for v, (m, n) in zip(X, mons):
        assert abs(v - quad_moment(m, n, -al, al)) < 1e-13
    aly, sy = np.arccos(b), np.sqrt(max(0.0, 1.0 - b * b))
    Y = [2 * aly, 0.0, 2 * sy, aly - b * sy, 0.0, aly + b * sy]
    for v, (m, n) in zip(Y, mons):
        assert abs(v - quad_moment(m, n, np.arcsin(b), np.pi - np.arcsin(b))) < 1e-13
    if a * a + b * b < 1.0:
        t0, t1 = np.arcsin(b), np.arccos(a)
        c0, s0, c1, s1 = sy, b, a, s  # end points (cos, sin)
        Q = [t1 - t0, s1 - s0, c0 - c1, 0.5 * (t1 - t0 + c1 * s1 - c0 * s0), 0.5 * (s1 * s1 - s0 * s0),
             0.5 * (t1 - t0 - c1 * s1 + c0 * s0)]
        for v, (m, n) in zip(Q, mons):
            assert abs(v - quad_moment(m, n, t0, t1)) < 1e-13
