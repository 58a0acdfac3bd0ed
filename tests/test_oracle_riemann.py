"""Pins of the exact Riemann solver (oracle/riemann.py), the analytic
reference of the Sod test, against what gas dynamics fixes: the
Rankine-Hugoniot conditions across every shock, the isentrope and the
Riemann invariant through every rarefaction fan, continuity of pressure and
velocity at the contact and of the fan at its head and tail, uniform states,
and mirror symmetry."""
import numpy as np

from oracle import riemann as R

G = 5.0 / 3.0
SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.125))


def rh_residuals(a, b, S, g=G):
    """Mass, momentum and energy flux jumps across a discontinuity moving at S
    between states a and b = (rho, u, p), relative to the fluxes."""
    out = []
    fl = []
    for rho, u, p in (a, b):
        w = u - S
        e = p / ((g - 1.0) * rho)
        fl.append((rho * w, rho * w * w + p, rho * w * (e + p / rho + 0.5 * w * w)))
    for k in range(3):
        out.append(abs(fl[0][k] - fl[1][k]) / max(abs(fl[0][k]), abs(fl[1][k]), 1e-300))
    return out


def states(left, right, g=G):
    ps, us = R.star(left, right, g)
    xi = np.linspace(-3, 3, 60001)
    rho, u, p = R.sample(xi, left, right, g)
    return ps, us, xi, rho, u, p


def jumps(xi, rho):
    return np.nonzero(np.abs(np.diff(rho)) > 1e-6 * np.max(rho))[0]


def test_sod_shock_satisfies_rankine_hugoniot():
    ps, us, xi, rho, u, p = states(*SOD)
    assert SOD[1][2] < ps < SOD[0][2] and us > 0
    # the right wave is a shock: star state just left of it, right state after
    right_star = (rho[(xi > us + 1e-3)][0], us, ps)
    Rr, ur, pr = SOD[1]
    S = (right_star[0] * us - Rr * ur) / (right_star[0] - Rr)     # mass flux fixes the speed
    assert S > us
    assert max(rh_residuals(right_star, SOD[1], S)) < 1e-12
    # and the sampled profile jumps exactly there
    k = np.argmin(np.abs(xi - S))
    assert abs(rho[k - 5] - right_star[0]) < 1e-12 and abs(rho[k + 5] - Rr) < 1e-12


def test_sod_rarefaction_is_isentropic_with_a_constant_riemann_invariant():
    ps, us, xi, rho, u, p = states(*SOD)
    rL, uL, pL = SOD[0]
    cL = np.sqrt(G * pL / rL)
    fan = (xi > uL - cL + 1e-6) & (xi < us - np.sqrt(G * ps / rho[xi < us][-1]) - 1e-6)
    assert fan.sum() > 1000
    c = np.sqrt(G * p[fan] / rho[fan])
    assert np.max(np.abs(p[fan] / rho[fan] ** G / (pL / rL ** G) - 1)) < 1e-12
    assert np.max(np.abs(u[fan] + 2 * c / (G - 1) - (uL + 2 * cL / (G - 1)))) < 1e-12
    assert np.allclose(u[fan] - c, xi[fan], atol=1e-12)          # on its own characteristic
    # continuous at the head and the tail
    assert np.max(np.abs(np.diff(p[(xi > uL - cL - 0.01) & (xi < us - 0.05)]))) < 1e-3


def test_contact_carries_pressure_and_velocity():
    for left, right in (SOD, ((1.0, 0.75, 1.0), (0.125, 0.0, 0.1)), ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4))):
        ps, us, xi, rho, u, p = states(left, right)
        a, b = xi < us - 1e-3, xi > us + 1e-3
        assert abs(p[a][-1] - ps) < 1e-12 and abs(p[b][0] - ps) < 1e-12
        assert abs(u[a][-1] - us) < 1e-12 and abs(u[b][0] - us) < 1e-12


def test_colliding_flows_make_two_shocks():
    left, right = (1.0, 1.5, 1.0), (0.5, -1.0, 0.8)
    ps, us, xi, rho, u, p = states(left, right)
    assert ps > left[2] and ps > right[2]
    for side, far in ((-1, left), (1, right)):
        star_rho = rho[(xi < us - 1e-3)][-1] if side < 0 else rho[(xi > us + 1e-3)][0]
        S = (star_rho * us - far[0] * far[1]) / (star_rho - far[0])
        assert (S < us) if side < 0 else (S > us)
        assert max(rh_residuals((star_rho, us, ps), far, S)) < 1e-12


def test_uniform_states_and_mirror_symmetry():
    st = (0.7, 0.3, 2.0)
    ps, us = R.star(st, st)
    assert abs(ps - 2.0) < 1e-13 and abs(us - 0.3) < 1e-13
    xi = np.linspace(-2, 2, 401)
    r1, u1, p1 = R.sample(xi, *SOD)
    (a, b) = SOD
    r2, u2, p2 = R.sample(-xi, (b[0], -b[1], b[2]), (a[0], -a[1], a[2]))
    sel = np.abs(np.abs(xi) - 1e-9) > 0
    assert np.allclose(r1, r2, atol=1e-13) and np.allclose(u1, -u2, atol=1e-13) and np.allclose(p1, p2, atol=1e-13)
