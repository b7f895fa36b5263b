"""The algorithmic flop counts behind the benchmark's roofline fraction, derived by hand from the
formulas (no GPU), independently of the oracle's counting scalar: each count is written below
as the sum of its terms, one flop per +, -, *, / and square root of the formula as the paper
states it (sign changes, |x| and comparisons free; rational constants such as 13/12 are given,
not computed), and must equal both the oracle's instrumented count and the benchmark's table.
"""
import pytest

import bench


def reconstruction():
    """One fifth-order reconstruction f^+_{i+1/2} with the WENO-ZN weights (Sec. 3)."""
    q = 3 * (3 + 2)                       # Eq. (4): q_k = three constant multiples, two adds, k = 0..2
    is0 = (1 + 2) + (2 + 2) + (4 + 1)     # Eq. (isjiang), IS_0: f_{i-2} - 2 f_{i-1} + f_i (1 mul, 2 adds);
    #                                       f_{i-2} - 4 f_{i-1} + 3 f_i (2 mul, 2 adds); 13/12 a a + 1/4 b b (4 mul, 1 add)
    is1 = (1 + 2) + 1 + (4 + 1)           # IS_1: second difference; f_{i-1} - f_{i+1}; the same combination
    is2 = is0                             # IS_2: the mirror image of IS_0
    tau5 = 1                              # Eq. (tau): |IS_0 - IS_2|, one subtraction
    tau8 = 6 + 1                          # Eq. (tau8): (f_{i-2} + f_{i+2}) - 4 (f_{i-1} + f_{i+1}) + 6 f_i (4 adds,
    #                                       2 mul), then squared
    C = (3 + 1 + 1) + 2                   # Eq. (function): (IS_0 + IS_2 - tau + eps) / (tau + eps), then A r r
    alpha = 3 * (1 + 1 + 1 + 1)           # Eq. (new): c_k (C + tau8 / (IS_k + eps)), k = 0..2
    normalise = 2 + 3 + (3 + 2)           # Eq. (3): sum of the alpha_k, omega_k = alpha_k / sum, sum omega_k q_k
    return q + is0 + is1 + is2 + tau5 + tau8 + C + alpha + normalise


def roe_state(nv):
    """Roe average between cells i and i+1 and the eigenvectors of the flux Jacobian there
    (Sec. 4.3 / 4.4: characteristic fields); the direction frame (rho, m_n[, m_t], E)."""
    avg = 2 + 1 + 1 + 1                   # (s_L u_L + s_R u_R) / (s_L + s_R): 2 mul, 2 adds, 1 div
    velocities = avg * (2 if nv == 4 else 1)
    H = avg
    q2 = 3 if nv == 4 else 1              # u^2 (+ v^2)
    c = 1 + 1 + 1 + 1 + 1                 # sqrt((gamma - 1)(H - q^2/2))
    b = (1 + 1 + 1) + 2                   # b1 = (gamma - 1)/c^2, b2 = q^2 b1 / 2
    if nv == 3:
        R = 1 + 1 + 2 + 2 + 2             # u - c, u + c, H - u c, u^2/2, H + u c
        L = (3 + 4 + 1) + (1 + 1) + (3 + 4 + 1)   # rows of the u -+ c fields (b2 +- u/c)/2, -(b1 u +- 1/c)/2, b1/2;
        #                                           the u field: 1 - b2, b1 u (and -b1 free)
    else:
        R = 1 + 1 + 2 + 1 + 2             # u - c, u + c, H - u c, q^2/2, H + u c (v, 1, 0 given)
        L = (3 + 4 + 2 + 1) + (1 + 1 + 1) + (3 + 4 + 2 + 1)   # the u -+ c rows gain -b1 v/2; the u row b1 v;
        #                                                        the shear row (-v, 0, 1, 0) is free
    return velocities + H + q2 + c + b + R + L


def interface(nv):
    """One numerical flux: Roe state, projection of the 5 + 5 split-flux stencil points onto
    the nv characteristic fields, both reconstructions per field and their sum, back-projection."""
    if nv == 1:
        return 2 * reconstruction() + 1
    projection = 2 * 5 * nv * (nv + nv)   # sides x points x fields x (nv mul + nv adds, from 0)
    recon = nv * (2 * reconstruction() + 1)
    back = nv * (nv + (nv - 1))           # F^ = R g^: nv mul, nv - 1 adds per component
    return roe_state(nv) + projection + recon + back


def cell_split(nv):
    """One cell's LF split fluxes h+- = (F +- alpha U)/2 and Roe ingredients, per sweep."""
    if nv == 1:
        return 1 + 2 * 3                  # f = a u; (f +- alpha u)/2
    prim = (1 + (1 if nv == 4 else 0)) + (2 + (3 if nv == 4 else 1)) + 3   # u = m/rho (v); rho (u^2 + v^2)/2;
    #                                                                         p = (gamma - 1)(E - kin)
    flux = 2 + (1 if nv == 4 else 0) + 2  # m u + p, (m_t u), u (E + p)
    split = nv * 2 * 3                    # (F_m +- alpha U_m)/2
    return prim + flux + split + 1 + 2    # sqrt(rho); H = (E + p)/rho


def speed(nv):
    """One cell's LF speed |u_n| + c (both directions in 2D): primitives, sqrt(gamma p/rho), add."""
    if nv == 1:
        return 0
    prim = (1 + (1 if nv == 4 else 0)) + (2 + (3 if nv == 4 else 1)) + 3
    one = prim + 3 + 1
    return one * (2 if nv == 4 else 1)


def difference(nv):
    """Eq. (2): -(F^_{i+1/2} - F^_{i-1/2})/dx per variable, and in 2D the y part subtracted."""
    return nv * 2 + (nv * 3 if nv == 4 else 0)


def rk3(nv):
    """Shu-Osher SSP-RK3 per variable and step: U1 = U + dt L (2); 3/4 U + 1/4 (U1 + dt L) (5);
    U/3 + 2/3 (U2 + dt L) (5)."""
    return nv * (2 + 5 + 5)


def cell_update(nv):
    per_stage = interface(nv) * (2 if nv == 4 else 1) + cell_split(nv) * (2 if nv == 4 else 1) + speed(nv) \
        + difference(nv)
    return 3 * per_stage + rk3(nv)


def test_hand_counts():
    assert reconstruction() == 85
    assert (interface(1), interface(3), interface(4)) == (171, 755, 1090)
    assert (cell_split(1), cell_split(3), cell_split(4)) == (7, 32, 42)
    assert (speed(3), speed(4)) == (11, 28)
    assert (difference(1), difference(3), difference(4)) == (2, 6, 20)
    assert (rk3(1), rk3(3), rk3(4)) == (12, 36, 48)
    assert (cell_update(1), cell_update(3), cell_update(4)) == (552, 2448, 6984)


def test_bench_tables_follow_the_derivation():
    assert bench.OPS_2D[(0, 0)] == (interface(4), cell_split(4), speed(4), difference(4), rk3(4))
    assert bench.OPS_1D == (interface(3), cell_split(3), speed(3), difference(3))
    assert bench.OPS_1D_CELL_UPDATE == cell_update(3)
    assert bench.RECON_FLOPS == reconstruction()
    fl = bench.algorithmic_flops(4096, 4096)
    assert fl["x_flux"] == interface(4) * 4097 * 4096 + cell_split(4) * 4096 * 4096
    assert fl["per_cell_update"] == pytest.approx(cell_update(4), rel=1e-3)    # plus the boundary interfaces


@pytest.mark.parametrize("system,nv", [(0, 1), (1, 3), (2, 4)])
def test_oracle_counter_agrees_with_the_derivation(orc, system, nv):
    parts = orc.opcount_parts(system)
    assert parts["interface"] == interface(nv)
    assert parts["cell_per_sweep"] == cell_split(nv)
    assert parts["wavespeed_cell"] == speed(nv)
