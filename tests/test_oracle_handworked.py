"""Hand-worked pins of the three oracle steps that no closed form of the paper
fixes on its own: the ghost value of Sec. 2.2.2, the doubly-unknown case of
the modified bounce-back (Sec. 2.2.2) and the (1/2) dG/dt history of Eq. BGK
(Sec. 2.1.3). Every expected number below is worked out in the comments from
the paper's definitions, independently of the oracle's code.

Lattice (paper order, Eq. ci): c_1 = (0,-1), c_2 = (1,0), c_3 = (0,1),
c_4 = (-1,0), c_5 = (1,1), c_6 = (-1,1), c_7 = (-1,-1), c_8 = (1,-1);
opposites 1<->3, 2<->4, 5<->7, 6<->8; w = 4/9, 1/9 (axes), 1/36 (diagonals);
c_s^2 = 1/3.
"""
import numpy as np

import oracle
from tests.oracle_fixtures import read_geometry


def phi_pattern(x, y):
    # the phi given to the zeta = 1 nodes of the ghost test: multiples of 1/8
    return ((x * x + 3 * y) % 8) / 8.0


def test_ghost_value_is_zeta_weighted_mean_of_3x3():
    # 7 x 6 lattice, periodic in x and y, solid block x = 1..5, y = 1..4.
    # The block's rim touches fluid: boundary (zeta = 1). Its inside, x = 2..4,
    # y = 2..3, has no fluid neighbour but a zeta = 1 one: six ghost nodes.
    # Sec. 2.2.2: a ghost takes sum_j zeta_j phi_j / sum_j zeta_j over its 3x3
    # neighbourhood (b = 9; zeta of the ghost itself is 0).
    nx, ny = 7, 6
    solid = np.zeros((ny, nx), np.uint8)
    solid[1:5, 1:6] = 1
    o = oracle.Oracle(solid, theta_deg=90.0, wrap_y=True)
    g = o.geometry()
    assert [(x, y) for y in range(ny) for x in range(nx) if g["cls"][y, x] == oracle.GHOST] == \
        [(2, 2), (3, 2), (4, 2), (2, 3), (3, 3), (4, 3)]
    xs, ys = np.meshgrid(np.arange(nx), np.arange(ny))
    o.init_phi(phi_pattern(xs, ys))
    phi, _, _ = o.get()
    # phi on the rim, (x,y): value = ((x^2 + 3y) mod 8)/8
    #   (1,1) 4/8  (2,1) 7/8  (3,1) 4/8  (4,1) 3/8  (5,1) 4/8
    #   (1,2) 7/8  (5,2) 7/8  (1,3) 2/8  (5,3) 2/8
    #   (1,4) 5/8  (2,4) 0    (3,4) 5/8  (4,4) 4/8  (5,4) 5/8
    # ghost (2,2): zeta=1 neighbours (1,1) (2,1) (3,1) (1,2) (1,3)
    #   = (4 + 7 + 4 + 7 + 2)/8 = 24/8 over 5 -> 3/5
    # ghost (3,2): (2,1) (3,1) (4,1) = (7 + 4 + 3)/8 = 14/8 over 3 -> 7/12
    # ghost (4,2): (3,1) (4,1) (5,1) (5,2) (5,3) = (4 + 3 + 4 + 7 + 2)/8 = 20/8 over 5 -> 1/2
    # ghost (2,3): (1,2) (1,3) (1,4) (2,4) (3,4) = (7 + 2 + 5 + 0 + 5)/8 = 19/8 over 5 -> 19/40
    # ghost (3,3): (2,4) (3,4) (4,4) = (0 + 5 + 4)/8 = 9/8 over 3 -> 3/8
    # ghost (4,3): (5,2) (5,3) (3,4) (4,4) (5,4) = (7 + 2 + 5 + 4 + 5)/8 = 23/8 over 5 -> 23/40
    # (dividing by 9 instead would give 1/3, 7/36, ...; axis neighbours only
    # would give 7/8, 1/2, 5/8, 1/8, 5/8, 3/8)
    expected = {(2, 2): 3 / 5, (3, 2): 7 / 12, (4, 2): 1 / 2,
                (2, 3): 19 / 40, (3, 3): 3 / 8, (4, 3): 23 / 40}
    for (x, y), v in expected.items():
        assert abs(phi[y, x] - v) < 1e-14, ((x, y), phi[y, x], v)
    # the rim keeps the values it was given (phi = sum_i g_i of g^eq)
    rim = (g["cls"] == oracle.BOUNDARY)
    assert np.max(np.abs(phi[rim] - phi_pattern(xs, ys)[rim])) < 1e-14


def test_doubly_unknown_link_takes_own_post_collision_opposite():
    # The 12 x 10 block-on-floor map of tests/golden/geometry_block.txt. Node
    # (2,1) is the boundary node at the foot of the block: the links c = (1,1)
    # (i = 5) and c = (-1,-1) (i = 7) are doubly unknown (zeta(x - c) =
    # zeta(x + c) = 0), the links (0,1) (i = 3), (-1,1) (i = 6) and (-1,0)
    # (i = 4) are unknown once.
    mask, _, _ = read_geometry("geometry_block.txt")
    ny, nx = mask.shape
    # rho_l = rho_g = 1 (grad rho = 0), tau_f = 1 (f* = f^eq + F_i),
    # theta = 90 deg (cos theta ~ 6e-17: no wall energy at this tolerance)
    o = oracle.Oracle(mask, theta_deg=90.0, sigma=0.01, W=4.0, M=0.1, tau_f=1.0,
                      rho_l=1.0, rho_g=1.0)
    zeta = o.geometry()["zeta"].astype(bool)
    f = np.zeros((9, ny, nx))
    g = np.zeros((9, ny, nx))
    # phi = sum_i g_i = 1/4 on every zeta = 1 node; the ghosts average to 1/4
    # too, so grad(phi) = lap(phi) = 0 everywhere and F = mu grad(phi) = 0:
    # F_i = 0 and f* = f^eq(p, u).
    g[0][zeta] = 0.25
    # node (2,1): f_2 = 0.03 (c = (1,0)), f_3 = 0.01 (c = (0,1)), the rest 0.
    #   u = sum c_i f_i / rho = (0.03, 0.01), u.u = 0.001, sum_{i!=0} f_i = 0.04
    #   s_0(u) = w_0 (-u.u / (2 c_s^2)) = (4/9)(-0.0015)
    #   p = c_s^2/(1 - w_0) [0.04 + 0 + rho s_0] = 0.6 (0.04 - 0.0006667) = 0.0236
    #   f^eq_i = w_i [p / c_s^2 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u], p / c_s^2 = 0.0708
    #   f*_7: c.u = -0.04 -> (0.0708 - 0.12 + 0.0072 - 0.0015)/36 = -0.0435/36
    #   f*_5: c.u = +0.04 -> (0.0708 + 0.12 + 0.0072 - 0.0015)/36 = 0.1965/36
    f[2, 1, 2] = 0.03
    f[3, 1, 2] = 0.01
    # node (2,2), directly above: f_2 = 0.02, the rest 0.
    #   u = (0.02, 0), u.u = 0.0004, p = 0.6 (0.02 - (4/9) 0.0006) = 0.01184
    #   f*_1 (c = (0,-1), c.u = 0) = (3 p - 1.5 u.u)/9 = (0.03552 - 0.0006)/9 = 0.00388
    f[2, 2, 2] = 0.02
    o.set_state(f, g)
    o.step(1)
    fa, _, _ = o.state()
    # doubly unknown: f_5(x) = f*_7(x) and f_7(x) = f*_5(x) of the node itself
    # (the post-streaming f_7(x) would come from x + c_5 = (3,2), a ghost)
    assert abs(fa[5, 1, 2] - (-0.0435 / 36)) < 1e-15, fa[5, 1, 2]
    assert abs(fa[7, 1, 2] - (0.1965 / 36)) < 1e-15, fa[7, 1, 2]
    # unknown once: f_3(x) = the post-streaming f_1(x) = f*_1 of (2,2)
    assert abs(fa[3, 1, 2] - 0.00388) < 1e-15, fa[3, 1, 2]
    # and f_1 itself streamed in from (2,2)
    assert abs(fa[1, 1, 2] - 0.00388) < 1e-15, fa[1, 1, 2]


def test_half_dG_dt_is_backward_difference_with_first_step_history():
    # 5 x 5 lattice, periodic in x and y, no solid: g*_i(x) is read back as
    # the post-streaming g_i(x + c_i) one step later. tau_g = 1 (the default),
    # so g*_i = g^eq_i + (source of Eq. BGK).
    nx = ny = 5
    o = oracle.Oracle(np.zeros((ny, nx), np.uint8), theta_deg=90.0, sigma=0.01, W=4.0, M=0.1,
                      tau_f=0.8, rho_l=1.0, rho_g=1.0, wrap_y=True)
    cx, cy, _, _ = oracle.lattice()
    # phi = 1/2 everywhere except phi(3,2) = 3/4 and phi(1,2) = 1/4, given
    # through g_0 (g_i = 0 for i != 0). At the node (2,2):
    #   lap(phi) = (2/3)(3/4 + 1/4 + 1/2 + 1/2) + (1/6)(4 * 1/2) - (10/3)(1/2) = 0
    #   mu = 4 beta (1/2)(-1/2)(0) - kappa * 0 = 0  ->  g^eq_0 = 1/2, g^eq_i = 0
    #   grad(phi) = ((3/4 - 1/4)/3, 0) = (1/6, 0)
    phi = np.full((ny, nx), 0.5)
    phi[2, 3] = 0.75
    phi[2, 1] = 0.25

    def state(m):
        # node (2,2) carries f_2 = m (c = (1,0)): rho = 1, F = mu grad(phi) = 0,
        # so u = (m, 0) and s = u.grad(phi) = m/6
        f = np.zeros((9, ny, nx))
        g = np.zeros((9, ny, nx))
        g[0] = phi
        f[2, 2, 2] = m
        return f, g

    def g_star():
        _, g, _ = o.state()
        out = np.zeros(9)
        out[0] = g[0, 2, 2]
        for i in range(1, 9):
            out[i] = g[i, (2 + cy[i]) % ny, (2 + cx[i]) % nx]
        return out

    # G_i(s) = w_i s h_i (Eq. F_i), h_0 = -2, h_axes = -1/2, h_diagonals = 1.
    # Step 1, m = 0.012: s(t) = 0.002. No history yet: s(t-1) = s(t), so
    # G(t) + (G(t) - G(t-1))/2 = G(s = 0.002):
    #   g*_0 = 1/2 + (4/9)(0.002)(-2) = 1/2 - 0.016/9
    #   g*_axis = (1/9)(0.002)(-1/2) = -0.001/9
    #   g*_diag = (1/36)(0.002) = 0.002/36
    # (taking s(t-1) = 0 instead would give 1.5x these sources)
    o.set_state(*state(0.012))
    o.step(1)
    gs = g_star()
    exp1 = np.array([0.5 - 0.016 / 9] + [-0.001 / 9] * 4 + [0.002 / 36] * 4)
    assert np.max(np.abs(gs - exp1)) < 1e-15, gs - exp1
    # Step 2 from the same phi, m = -0.024: s(t) = -0.004, s(t-1) = 0.002.
    # 1.5 G(s(t)) - 0.5 G(s(t-1)) = w h (1.5 (-0.004) - 0.5 (0.002)) = -0.007 w h:
    #   g*_0 = 1/2 + (4/9)(-0.007)(-2) = 1/2 + 0.056/9
    #   g*_axis = (1/9)(-0.007)(-1/2) = 0.0035/9
    #   g*_diag = (1/36)(-0.007) = -0.007/36
    # (dropping the term gives -0.004 w h; swapping t and t-1 gives +0.005 w h)
    o.set_state(*state(-0.024))
    o.step(1)
    gs = g_star()
    exp2 = np.array([0.5 + 0.056 / 9] + [0.0035 / 9] * 4 + [-0.007 / 36] * 4)
    assert np.max(np.abs(gs - exp2)) < 1e-15, gs - exp2
