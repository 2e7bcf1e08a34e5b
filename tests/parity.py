"""Error measures shared by the parity tests and bench.py.

Relative L1 error per conserved field (the reading used throughout): for
each conserved quantity of the governing equations (Sect. 2.1: mass, momentum
vector, energy; and dust mass, dust momentum vector),

    err = sum_cells V |q_test - q_ref|_1 / sum_cells V |q_ref|_1,

where |.|_1 of the momentum is the sum of the absolute values of its three
components.  The per-component ratios and the same measure on the
deviations from equilibrium are reported alongside (they are stricter: the
radial and vertical momenta vanish at equilibrium).
"""
import numpy as np

GROUPS = {
    "mass": (4,),
    "momentum": (0, 1, 2),
    "energy": (3,),
    "dust_mass": (8,),
    "dust_momentum": (5, 6, 7),
}


def rel_l1(E_test, E_ref, V):
    """E arrays (nf, nz, nth, nr) float64; V (nr,) cell volumes. Returns {group: err}."""
    nf = E_ref.shape[0]
    Vb = V[None, None, :]
    out = {}
    for name, fields in GROUPS.items():
        if max(fields) >= nf:
            continue
        num = sum((Vb * np.abs(E_test[f] - E_ref[f])).sum() for f in fields)
        den = sum((Vb * np.abs(E_ref[f])).sum() for f in fields)
        out[name] = float(num / den) if den > 0 else float(num)
    return out


def rel_l1_components(E_test, E_ref, V, E0=None):
    """Per-field relative L1 (on deviations from E0 when given)."""
    Vb = V[None, None, :]
    out = []
    for f in range(E_ref.shape[0]):
        a, b = E_test[f], E_ref[f]
        if E0 is not None and f < 5:
            a = a - E0[f][:, None, :]
            b = b - E0[f][:, None, :]
        den = (Vb * np.abs(b)).sum()
        num = (Vb * np.abs(a - b)).sum()
        out.append(float(num / den) if den > 0 else float(num))
    return out


def jitter(E, gamma, rng, a):
    """A state near E away from exact ties of the limiter: relative noise a on
    rho, P and rho_d, and a * c_s on the gas and dust velocities."""
    E = E.copy()
    rho = E[4]
    v = E[0:3] / rho
    P = (gamma - 1.0) * (E[3] - 0.5 * (E[0:3] ** 2).sum(0) / rho)
    cs = np.sqrt(gamma * P / rho)
    rho2 = rho * (1.0 + a * rng.standard_normal(rho.shape))
    P2 = P * (1.0 + a * rng.standard_normal(rho.shape))
    v2 = v + a * cs * rng.standard_normal(v.shape)
    E[4] = rho2
    E[0:3] = rho2 * v2
    E[3] = P2 / (gamma - 1.0) + 0.5 * rho2 * (v2 ** 2).sum(0)
    if E.shape[0] > 5:
        rd = E[8] * (1.0 + a * rng.standard_normal(rho.shape))
        vd = E[5:8] / E[8] + a * cs * rng.standard_normal(v.shape)
        E[8] = rd
        E[5:8] = rd * vd
    return E


def elementwise(E_test, E_ref, E0=None):
    """Element-wise error per conserved quantity (the groups of GROUPS): the
    largest |q_test - q_ref| over cells and components, divided by the
    largest departure |q_ref - q0| of the group (q0 = E0 for the gas, 0 for
    the dust; the largest |q_ref| when there is no E0).  Returns
    {group: (ratio, (field, k, j, i) of the largest difference)}.  Unlike the
    L1 measure it cannot average a single bad cell (a tile edge, a ghost)
    away."""
    nf = E_ref.shape[0]
    out = {}
    for name, fields in GROUPS.items():
        if max(fields) >= nf:
            continue
        num, where, den = -1.0, None, 0.0
        for f in fields:
            d = np.abs(E_test[f] - E_ref[f])
            idx = np.unravel_index(int(np.argmax(d)), d.shape)
            if d[idx] > num:
                num, where = float(d[idx]), (f,) + tuple(int(v) for v in idx)
            dep = E_ref[f] - (E0[f][:, None, :] if (E0 is not None and f < 5) else 0.0)
            den = max(den, float(np.abs(dep).max()))
        out[name] = (num / den if den > 0 else num, where)
    return out
