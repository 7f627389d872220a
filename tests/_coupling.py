"""The caller's side of the radiation-gas coupling for the sec. 5.2 moving
medium test: a uniform, periodic medium has no gas fluxes, so the MHD update
(Steps 6-7 of sec. 4.1) reduces to adding the radiation sources, momentum
rho v += Delta(rho v), and taking the new gas temperature of the implicit
energy exchange.  `step(v, T)` advances the radiation one step with the given
gas state and returns (E, F, P, dMom, T_new); the same loop drives the oracle
and the GPU library."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_values():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_values.txt")) as f:
        for line in f:
            if not line.startswith("#") and line.strip():
                k, v = line.split()[:2]
                vals[k] = float(v)
    return vals


def drag_history(step, nsteps, rho, T, v, E0, F0, C, P, kv):
    """Runs nsteps coupled steps; returns per-step dicts with E, F, P, v, T
    and the relative changes of the total momentum rho v_x + P F_x / C and
    of the total energy rho v^2 / 2 + kv rho T + P E_r (per cell)."""
    mom0 = rho * v[0] + P * F0[0] / C
    en0 = 0.5 * rho * (v ** 2).sum(axis=0) + kv * rho * T + P * E0
    hist = []
    for _ in range(nsteps):
        E, F, Pm, dMom, T = step(v, T)
        v = v + dMom / rho
        mom = rho * v[0] + P * F[0] / C
        en = 0.5 * rho * (v ** 2).sum(axis=0) + kv * rho * T + P * E
        hist.append(dict(E=E, F=F, P=Pm, v=v.copy(), T=T.copy(), dmom=np.abs(mom - mom0).max() / np.abs(mom0).max(),
                         den=np.abs(en - en0).max() / np.abs(en0).max()))
    return hist
