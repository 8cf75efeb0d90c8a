"""Closed-form deflection and deformation tensor per component (oracle, FP64).

TEST INFRASTRUCTURE ONLY.

Conventions (Sec. 2.1): angles in arcsec (theta_0 = 1"), the potential psi is
defined without a_dis, so every strength here is the a_dis = 1 value; the
position angle is counter-clockwise from +x; ellipticity eps = (1-q)/(1+q).
Each function takes offsets (dx, dy) = theta - theta_c as float64 tensors (any
broadcastable shape, e.g. (S, 1) parameters against (1, N) positions) and
returns (alpha_x, alpha_y, psi_xx, psi_yy, psi_xy).

The paper lists no profile formulas; it follows Keeton (2001) for the PJE
(Sec. 3.4) and names an "isothermal ellipsoid with a finite core radius"
(SIELens, Sec. 5).  The forms below are that catalogue's softened isothermal
ellipsoid, its dPIE difference, the spherical NFW (Bartelmann 1996) and the
external shear, written from their definitions.  Pins: tests/test_oracle_profiles.py.
"""
import torch


def _rotate_back(c, s, au, av, puu, pvv, puv):
    """(u, v) = M (dx, dy) with M = [[c, s], [-s, c]]: alpha = M^T alpha_uv,
    Psi = M^T Psi_uv M."""
    ax = c * au - s * av
    ay = s * au + c * av
    pxx = c * c * puu - 2.0 * c * s * puv + s * s * pvv
    pyy = s * s * puu + 2.0 * c * s * puv + c * c * pvv
    pxy = c * s * (puu - pvv) + (c * c - s * s) * puv
    return ax, ay, pxx, pyy, pxy


def sie(dx, dy, b, q, pa, s):
    """Cored (softened) isothermal ellipsoid.

    kappa = (b/2) / sqrt(s^2 + u^2 + v^2/q^2) with (u, v) the frame rotated by
    the position angle (major axis along u).  With psi~ = sqrt(q^2 (s^2 + u^2) + v^2)
    and e = sqrt(1 - q^2):
      alpha_u = (b q / e) atan(e u / (psi~ + s)),
      alpha_v = (b q / e) atanh(e v / (psi~ + q^2 s)),
      psi_uu = (b q / psi~) (q^2 s^2 + v^2 + s psi~) / D,
      psi_vv = (b q / psi~) (s^2 + u^2 + s psi~) / D,
      psi_uv = -(b q / psi~) u v / D,    D = (1 + q^2) s^2 + 2 psi~ s + u^2 + v^2.
    q = 1 takes the limit alpha = b (u, v) / (psi~ + s), written to first order in
    e^2 = 1 - q^2 from the Taylor series of atan and atanh,
      alpha_u = b q X (1 - e^2 X^2 / 3),  alpha_v = b q Y (1 + e^2 Y^2 / 3),
      X = u / (psi~ + s),  Y = v / (psi~ + q^2 s),
    whose value is the limit and whose derivative in q there is exact (the next terms are
    O(e^4)), so that autograd through the round branch differentiates in eps correctly.
    """
    dx, dy, b, q, pa, s = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                                     for t in (dx, dy, b, q, pa, s)])
    c, sn = torch.cos(pa), torch.sin(pa)
    u = c * dx + sn * dy
    v = -sn * dx + c * dy
    q2 = q * q
    psi = torch.sqrt(q2 * (s * s + u * u) + v * v)
    e2 = (1.0 - q) * (1.0 + q)
    round_ = e2 == 0
    # the square root only of e^2 > 0 (its derivative at 0 is infinite)
    e_safe = torch.sqrt(torch.where(round_, torch.ones_like(e2), e2))
    au_ell = b * q / e_safe * torch.atan(e_safe * u / (psi + s))
    av_ell = b * q / e_safe * torch.atanh(e_safe * v / (psi + q2 * s))
    X, Y = u / (psi + s), v / (psi + q2 * s)
    au = torch.where(round_, b * q * X * (1.0 - e2 * X * X / 3.0), au_ell)
    av = torch.where(round_, b * q * Y * (1.0 + e2 * Y * Y / 3.0), av_ell)
    D = (1.0 + q2) * s * s + 2.0 * psi * s + u * u + v * v
    f = b * q / (psi * D)
    puu = f * (q2 * s * s + v * v + s * psi)
    pvv = f * (s * s + u * u + s * psi)
    puv = -f * u * v
    return _rotate_back(c, sn, au, av, puu, pvv, puv)


def dpie(dx, dy, b, q, pa, core, cut):
    """Pseudo-Jaffe ellipsoid / dPIE: the cored ellipsoid of core radius `core`
    minus the same ellipsoid of core radius `cut` (Keeton 2001), i.e.
    kappa = (b/2) [1/sqrt(core^2 + xi^2) - 1/sqrt(cut^2 + xi^2)], xi^2 = u^2 + v^2/q^2."""
    a1 = sie(dx, dy, b, q, pa, core)
    a2 = sie(dx, dy, b, q, pa, cut)
    return tuple(p - m for p, m in zip(a1, a2))


def cse_uv(u, v, q, s):
    """Unit cored steep ellipsoid (CSE) in its (u, v) frame: kappa = 1 / (2 (s^2 + xi^2)^(3/2)),
    xi^2 = u^2 + v^2/q^2.  This density is -(1/s) d/ds of the unit cored isothermal ellipsoid
    kappa = 1 / (2 sqrt(s^2 + xi^2)) of sie(), so its deflection is -(1/s) d alpha_sie / ds;
    the atan / atanh drop out and, with P = sqrt(q^2 (s^2 + u^2) + v^2),
    D = (1 + q^2) s^2 + 2 P s + u^2 + v^2, A = P + q^2 s, B = P + s:
      alpha_u = q u A / (s P D),  alpha_v = q v B / (s P D),
      psi_uu = q / (s P D) [A - q^4 s u^2 / P^2 - 2 u^2 A^2 / (P D)],
      psi_vv = q / (s P D) [B - s v^2 / P^2 - 2 v^2 B^2 / (P D)],
      psi_uv = -q u v / (s P D) [q^2 s / P^2 + 2 A B / (P D)].
    Valid at q = 1 as written.  Arguments broadcast."""
    q2 = q * q
    P = torch.sqrt(q2 * (s * s + u * u) + v * v)
    D = (1.0 + q2) * s * s + 2.0 * P * s + u * u + v * v
    A, B = P + q2 * s, P + s
    f = q / (s * P * D)
    au, av = f * u * A, f * v * B
    iP2, PD = 1.0 / (P * P), P * D
    puu = f * (A - q2 * q2 * s * u * u * iP2 - 2.0 * u * u * A * A / PD)
    pvv = f * (B - s * v * v * iP2 - 2.0 * v * v * B * B / PD)
    puv = -f * u * v * (q2 * s * iP2 + 2.0 * A * B / PD)
    return au, av, puu, pvv, puv


def enfw(dx, dy, ks, q, pa, rs, s_tab, a_tab):
    """Elliptical NFW of scale radius rs approximated by a CSE sum (Oguri 2021):
    kappa = 2 ks sum_i a_i / (2 (s_i^2 + xi^2 / rs^2)^(3/2)), xi^2 = u^2 + v^2/q^2, so
    alpha = 2 ks rs sum_i a_i alpha_cse(u/rs, v/rs; s_i) and Psi = 2 ks sum_i a_i Psi_cse.
    (s_tab, a_tab): the coefficient table (oracle.cse_nfw.table())."""
    dx, dy, ks, q, pa, rs = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                                      for t in (dx, dy, ks, q, pa, rs)])
    c, sn = torch.cos(pa), torch.sin(pa)
    u = (c * dx + sn * dy) / rs
    v = (-sn * dx + c * dy) / rs
    st = torch.as_tensor(s_tab, dtype=torch.float64)
    at = torch.as_tensor(a_tab, dtype=torch.float64)
    terms = cse_uv(u[..., None], v[..., None], q[..., None], st)
    au, av, puu, pvv, puv = [(t * at).sum(-1) for t in terms]
    k2 = 2.0 * ks
    return _rotate_back(c, sn, k2 * rs * au, k2 * rs * av, k2 * puu, k2 * pvv, k2 * puv)


def _axisym(dx, dy, kbar, kappa, r2):
    """Axially symmetric lens: alpha = kbar (dx, dy) with kbar the mean convergence
    inside r, Psi_ij = kbar delta_ij + 2 (kappa - kbar) x_i x_j / r^2."""
    pos = r2 > 0
    r2s = torch.where(pos, r2, torch.ones_like(r2))
    t = torch.where(pos, 2.0 * (kappa - kbar) / r2s, torch.zeros_like(r2))
    return kbar * dx, kbar * dy, kbar + t * dx * dx, kbar + t * dy * dy, t * dx * dy


def pje_sph(dx, dy, b, core, cut):
    """Spherical pseudo-Jaffe (dPIE with q = 1), used for cluster members under axial
    symmetry (Sec. 4.1, 4.2).  With S = sqrt(core^2 + r^2), R = sqrt(cut^2 + r^2):
    kappa = (b/2)(1/S - 1/R), kbar = b/(S + core) - b/(R + cut)."""
    dx, dy, b, core, cut = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                                     for t in (dx, dy, b, core, cut)])
    r2 = dx * dx + dy * dy
    S = torch.sqrt(core * core + r2)
    R = torch.sqrt(cut * cut + r2)
    kbar = b / (S + core) - b / (R + cut)
    kappa = 0.5 * b * (1.0 / S - 1.0 / R)
    return _axisym(dx, dy, kbar, kappa, r2)


def _series(w, n_terms=12):
    """sum_{n>=0} w^n / (2n + 1)  (= atanh(sqrt w)/sqrt w for w > 0, atan(sqrt -w)/sqrt -w for w < 0)."""
    out = torch.zeros_like(w)
    p = torch.ones_like(w)
    for n in range(n_terms):
        out = out + p / (2 * n + 1)
        p = p * w
    return out


def nfw_sph(dx, dy, ks, rs):
    """Spherical NFW (Bartelmann 1996) with x = r / rs:
    F(x) = atanh(sqrt(1-x^2))/sqrt(1-x^2) (x<1), atan(sqrt(x^2-1))/sqrt(x^2-1) (x>1);
    kappa = 2 ks (1 - F)/(x^2 - 1);  h(x) = ln(x/2) + 2 atanh(sqrt((1-x)/(1+x)))/sqrt(1-x^2)
    (atan form for x > 1);  kbar = 4 ks h / x^2.  Near x = 1 both use the power series
    in w = 1 - x^2 and u = (1-x)/(1+x) of the same functions."""
    dx, dy, ks, rs = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                               for t in (dx, dy, ks, rs)])
    r2 = dx * dx + dy * dy
    x2 = r2 / (rs * rs)
    x = torch.sqrt(x2)
    w = (1.0 - x) * (1.0 + x)
    near = w.abs() < 1e-3
    lt = (w > 0) & ~near
    gt = (w < 0) & ~near
    wl = torch.where(lt, w, torch.full_like(w, 0.5))
    wg = torch.where(gt, -w, torch.full_like(w, 0.5))
    Flt = torch.atanh(torch.sqrt(wl)) / torch.sqrt(wl)
    Fgt = torch.atan(torch.sqrt(wg)) / torch.sqrt(wg)
    # (1 - F)/(x^2 - 1) = (F - 1)/w ; near x = 1 the series sum_{n>=1} w^{n-1}/(2n+1)
    g_near = _tail(torch.where(near, w, torch.zeros_like(w)))
    F = torch.where(lt, Flt, torch.where(gt, Fgt, torch.ones_like(w)))
    wsafe = torch.where(near, torch.ones_like(w), w)
    kappa = 2.0 * ks * torch.where(near, g_near, (F - 1.0) / wsafe)
    # h(x) = ln(x/2) + (2/(1+x)) sum_n u^n/(2n+1), u = (1-x)/(1+x)
    u = (1.0 - x) / (1.0 + x)
    nu = u.abs() < 1e-3
    ul = torch.where((u > 0) & ~nu, u, torch.full_like(u, 0.5))
    ug = torch.where((u < 0) & ~nu, -u, torch.full_like(u, 0.5))
    Hl = torch.atanh(torch.sqrt(ul)) / torch.sqrt(ul)
    Hg = torch.atan(torch.sqrt(ug)) / torch.sqrt(ug)
    Hs = _series(torch.where(nu, u, torch.zeros_like(u)))
    Hsum = torch.where(nu, Hs, torch.where(u > 0, Hl, Hg))
    h = torch.log(x / 2.0) + 2.0 / (1.0 + x) * Hsum
    # Toward the centre the two terms cancel (h ~ x^2 ln(2/x) / 2 while each is ~ ln(2/x)).  For
    # x < 1, 2 atanh(sqrt(u)) = ln((1 + s)/x) with s = sqrt(1 - x^2), and 1 - s = d = x^2/(1 + s),
    # so h = [s ln(x/2) + ln((1 + s)/x)] / s = [d ln(2/x) + ln(1 - d/2)] / s, free of it.
    sm = (x < 0.5) & (x > 0)
    xs = torch.where(sm, x, torch.full_like(x, 0.25))
    sq = torch.sqrt((1.0 - xs) * (1.0 + xs))
    d = xs * xs / (1.0 + sq)
    h = torch.where(sm, (d * torch.log(2.0 / xs) + torch.log1p(-0.5 * d)) / sq, h)
    kbar = 4.0 * ks * h / x2
    return _axisym(dx, dy, kbar, kappa, r2)


def _tail(w, n_terms=12):
    """sum_{n>=1} w^{n-1} / (2n + 1) = (F - 1)/w for the series F above."""
    out = torch.zeros_like(w)
    p = torch.ones_like(w)
    for n in range(1, n_terms + 1):
        out = out + p / (2 * n + 1)
        p = p * w
    return out


def shear(dx, dy, gamma, pa):
    """External shear psi = (gamma/2) r^2 cos 2(phi - pa):
    (gamma1, gamma2) = gamma (cos 2pa, sin 2pa), alpha = (g1 dx + g2 dy, g2 dx - g1 dy),
    kappa = 0."""
    dx, dy, gamma, pa = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                                  for t in (dx, dy, gamma, pa)])
    g1 = gamma * torch.cos(2.0 * pa)
    g2 = gamma * torch.sin(2.0 * pa)
    return g1 * dx + g2 * dy, g2 * dx - g1 * dy, g1, -g1, g2


def mass_sheet(dx, dy, k0):
    """A uniform sheet of convergence k0 (oracle-only test profile): psi = k0 r^2 / 2, so
    alpha = k0 (dx, dy), psi_xx = psi_yy = k0, psi_xy = 0."""
    dx, dy, k0 = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64) for t in (dx, dy, k0)])
    return k0 * dx, k0 * dy, k0.clone(), k0.clone(), torch.zeros_like(k0)


def multipole3(dx, dy, amp, pa):
    """Third-order multipole whose potential grows as theta^2 (Sec. 4.2):
    psi = amp r^2 cos 3(phi - pa), phi the polar angle of (dx, dy).  From the polar
    derivatives psi_rr = 2 amp cos 3D, psi_r / r + psi_phiphi / r^2 = -7 amp cos 3D and
    d(psi_phi / r)/dr = -3 amp sin 3D (D = phi - pa), rotated to (x, y); kappa is
    -(5/2) amp cos 3D at every radius.  At r = 0 exactly everything is set to 0."""
    dx, dy, amp, pa = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                                for t in (dx, dy, amp, pa)])
    r = torch.hypot(dx, dy)
    phi = torch.atan2(dy, dx)
    c3, s3 = torch.cos(3.0 * (phi - pa)), torch.sin(3.0 * (phi - pa))
    a_r = 2.0 * amp * r * c3
    a_phi = -3.0 * amp * r * s3
    c, s = torch.cos(phi), torch.sin(phi)
    ax = a_r * c - a_phi * s
    ay = a_r * s + a_phi * c
    p_rr = 2.0 * amp * c3
    p_tt = -7.0 * amp * c3
    p_rt = -3.0 * amp * s3
    pxx = p_rr * c * c - 2.0 * p_rt * s * c + p_tt * s * s
    pyy = p_rr * s * s + 2.0 * p_rt * s * c + p_tt * c * c
    pxy = (p_rr - p_tt) * s * c + p_rt * (c * c - s * s)
    zero = r == 0
    out = [ax, ay, pxx, pyy, pxy]
    return tuple(torch.where(zero, torch.zeros_like(v), v) for v in out)


# ------------------------------------------------------------------ potentials ----
# The lens potential psi of each profile (up to a constant), needed by the time delay
# (Eq. time_delay).  Pins: grad psi = alpha (tests/test_oracle_potentials.py).

def sie_potential(dx, dy, b, q, pa, s):
    """Cored isothermal ellipsoid (Keeton 2001): in the (u, v) frame of sie(),
    psi = u alpha_u + v alpha_v - b q s ln sqrt((psi~ + s)^2 + (1 - q^2) u^2)."""
    dx, dy, b, q, pa, s = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                                     for t in (dx, dy, b, q, pa, s)])
    ax, ay, *_ = sie(dx, dy, b, q, pa, s)
    c, sn = torch.cos(pa), torch.sin(pa)
    u = c * dx + sn * dy
    psit = torch.sqrt(q * q * (s * s + u * u) + (-sn * dx + c * dy) ** 2)
    lg = 0.5 * torch.log((psit + s) ** 2 + (1.0 - q * q) * u * u)
    return dx * ax + dy * ay - b * q * s * lg


def dpie_potential(dx, dy, b, q, pa, core, cut):
    return sie_potential(dx, dy, b, q, pa, core) - sie_potential(dx, dy, b, q, pa, cut)


def pje_sph_potential(dx, dy, b, core, cut):
    """Round pseudo-Jaffe: psi = b [(S - core ln(S + core)) - (R - cut ln(R + cut))], whose
    radial derivative is b r [1/(S + core) - 1/(R + cut)]."""
    dx, dy, b, core, cut = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                                     for t in (dx, dy, b, core, cut)])
    r2 = dx * dx + dy * dy
    S = torch.sqrt(core * core + r2)
    R = torch.sqrt(cut * cut + r2)
    return b * ((S - core * torch.log(S + core)) - (R - cut * torch.log(R + cut)))


def nfw_potential(dx, dy, ks, rs):
    """Spherical NFW: psi = 2 ks rs^2 [ln^2(x/2) - atanh^2 sqrt(1 - x^2)] (x < 1),
    [ln^2(x/2) + atan^2 sqrt(x^2 - 1)] (x > 1), ln^2(1/2) at x = 1; its derivative in x is
    4 ks rs h(x)/x as in nfw_sph().  For x < 1, atanh sqrt(1 - x^2) = ln((1 + w)/x) with
    w = sqrt(1 - x^2), and the difference of squares is evaluated as the product
    ln(x^2 / (2 (1 + w))) ln((1 + w) / 2), free of the cancellation of the two squares."""
    dx, dy, ks, rs = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                               for t in (dx, dy, ks, rs)])
    x = torch.sqrt(dx * dx + dy * dy) / rs
    w2 = (1.0 - x) * (1.0 + x)
    lt = w2 > 0
    w = torch.sqrt(torch.where(lt, w2, torch.zeros_like(w2)))
    g_lt = torch.log(x * x / (2.0 * (1.0 + w))) * torch.log((1.0 + w) / 2.0)
    wg = torch.where(~lt, -w2, torch.zeros_like(w2))
    g_gt = torch.log(x / 2.0) ** 2 + torch.atan(torch.sqrt(wg)) ** 2
    return 2.0 * ks * rs * rs * torch.where(lt, g_lt, g_gt)


def cse_potential_uv(u, v, q, s):
    """Unit CSE potential: -(1/s) d/ds of the cored isothermal potential
    u alpha_u + v alpha_v - q s ln sqrt(D) (sie_potential),
      u alpha_u + v alpha_v + (q / (2 s)) ln D + (q / (2 D)) dD/ds,
    dD/ds = 2 (1 + q^2) s + 2 P + 2 q^2 s^2 / P, less its value at the centre,
    (q / (2 s)) ln((1 + q)^2 s^2) + q / s (there P = q s, D = (1 + q)^2 s^2), so that psi(0) = 0:
      u alpha_u + v alpha_v + (q / (2 s)) ln(D / ((1 + q)^2 s^2))
        - q [s (q^2 u^2 + v^2) / P + u^2 + v^2] / (s D)."""
    q2 = q * q
    P = torch.sqrt(q2 * (s * s + u * u) + v * v)
    D = (1.0 + q2) * s * s + 2.0 * P * s + u * u + v * v
    au, av = cse_uv(u, v, q, s)[:2]
    return (u * au + v * av + q / (2.0 * s) * torch.log(D / ((1.0 + q) ** 2 * s * s))
            - q * (s * (q2 * u * u + v * v) / P + u * u + v * v) / (s * D))


def enfw_potential(dx, dy, ks, q, pa, rs, s_tab, a_tab):
    """psi = 2 ks rs^2 sum_i a_i psi_cse(u/rs, v/rs; s_i) (the potential scales as length^2)."""
    dx, dy, ks, q, pa, rs = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                                      for t in (dx, dy, ks, q, pa, rs)])
    c, sn = torch.cos(pa), torch.sin(pa)
    u = (c * dx + sn * dy) / rs
    v = (-sn * dx + c * dy) / rs
    st = torch.as_tensor(s_tab, dtype=torch.float64)
    at = torch.as_tensor(a_tab, dtype=torch.float64)
    p = (cse_potential_uv(u[..., None], v[..., None], q[..., None], st) * at).sum(-1)
    return 2.0 * ks * rs * rs * p


def shear_potential(dx, dy, gamma, pa):
    """psi = (gamma/2) r^2 cos 2(phi - pa) = (g1 (x^2 - y^2) + 2 g2 x y) / 2."""
    dx, dy, gamma, pa = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                                  for t in (dx, dy, gamma, pa)])
    g1, g2 = gamma * torch.cos(2.0 * pa), gamma * torch.sin(2.0 * pa)
    return 0.5 * g1 * (dx * dx - dy * dy) + g2 * dx * dy


def mass_sheet_potential(dx, dy, k0):
    """psi = k0 r^2 / 2."""
    dx, dy, k0 = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64) for t in (dx, dy, k0)])
    return 0.5 * k0 * (dx * dx + dy * dy)


def multipole3_potential(dx, dy, amp, pa):
    """psi = amp r^2 cos 3(phi - pa), the definition."""
    dx, dy, amp, pa = torch.broadcast_tensors(*[torch.as_tensor(t, dtype=torch.float64)
                                                for t in (dx, dy, amp, pa)])
    return amp * (dx * dx + dy * dy) * torch.cos(3.0 * (torch.atan2(dy, dx) - pa))

