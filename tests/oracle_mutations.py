"""Checks that the oracle's pins catch plausible mistakes in the oracle.

Each entry below alters oracle/rt_oracle.c in one plausible way (a dropped
factor, a flipped sign, a wrong upwind side, a step counted in the wrong
place), builds the altered copy in a temporary folder (the repository's
files are not touched: RT_ORACLE_SRC / RT_ORACLE_LIB point the oracle module
at the copy) and runs the oracle's pin tests against it.  Every alteration
must make at least one pin fail; the script prints the first failing pin of
each and exits 1 if any alteration survives.

usage: python tests/oracle_mutations.py [name ...]     (about six minutes for all on eight cores)
"""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "rt_oracle.c")
PINS = ["test_oracle_angles.py", "test_oracle_transport.py", "test_oracle_sources.py", "test_oracle_sec5.py",
        "test_oracle_bf16.py"]

# name -> [(text in rt_oracle.c, replacement), ...]
MUTATIONS = {
    # van Leer slope and face states (sec. 4.2)
    "slope without its factor 2": [("return pr > 0 ? 2.0 * pr / (dl + dr) : 0.0;", "return pr > 0 ? pr / (dl + dr) : 0.0;")],
    "slope not limited": [("return pr > 0 ? 2.0 * pr / (dl + dr) : 0.0;", "return 0.5 * (dl + dr);")],
    "Courant number without alpha": [("double nu = af * p->C * fabs(mud) * rdx;", "double nu = p->C * fabs(mud) * rdx;")],
    "face states not time-centred": [("double left = It[qa] + 0.5 * (1.0 - nu) * sa;", "double left = It[qa] + 0.5 * sa;"),
                                     ("double right = It[qb] - 0.5 * (1.0 - nu) * sb;", "double right = It[qb] - 0.5 * sb;")],
    "alpha weights on the wrong sides": [("0.5 * (1.0 + af) * up + 0.5 * (1.0 - af) * down",
                                          "0.5 * (1.0 - af) * up + 0.5 * (1.0 + af) * down")],
    "upwind side reversed": [("double up = mud > 0 ? left : right, down = mud > 0 ? right : left;",
                              "double up = mud > 0 ? right : left, down = mud > 0 ? left : right;")],
    "alpha of one cell at a face": [("double af = 0.5 * (al[qa] + al[qb]);", "double af = al[qa];")],
    "alpha without its factor 10": [("double s = 10.0 * dl * sigma_t;", "double s = dl * sigma_t;")],
    # the IV term (eqs. decomposeI, transporttwoterms)
    "IV taken downwind": [("double ivf = vf > 0 ? lv : (vf < 0 ? rv : 0.5 * (lv + rv));",
                           "double ivf = vf > 0 ? rv : (vf < 0 ? lv : 0.5 * (lv + rv));")],
    "IV flux with the wrong sign": [("fl[f] = fI + mud * ivf;", "fl[f] = fI - mud * ivf;")],
    "I~ = I + IV/C": [("It[q] = intensity_at(p, I, m, c, d, j) - iv / p->C;",
                       "It[q] = intensity_at(p, I, m, c, d, j) + iv / p->C;")],
    "IV without its factor 3": [("double iv = 3.0 * (nm[0]", "double iv = 1.0 * (nm[0]")],
    "IV faces not time-centred": [("double lv = IV[qa] + 0.5 * (1.0 - nv) * va;", "double lv = IV[qa] + 0.5 * va;"),
                                  ("double rv = IV[qb] - 0.5 * (1.0 - nv) * vb;", "double rv = IV[qb] - 0.5 * vb;")],
    "one axis's cell size for all": [("double rdx = dt / p->dx[d];", "double rdx = dt / p->dx[0];")],
    "IV face velocity of one cell": [("double vf = 0.5 * (vd[qa] + vd[qb]);", "double vf = vd[qa];")],
    "IV Courant number times C": [("double nv = fabs(vf) * rdx;", "double nv = fabs(vf) * rdx * p->C;")],
    "opacity without scattering": [("    J[c] = E[c] / (4 * ORC_PI);\n    st[c] = sa[c] + ss[c];",
                                    "    J[c] = E[c] / (4 * ORC_PI);\n    st[c] = sa[c];")],
    # quadrature (sec. 3) and the step-n moments the step uses
    "P_xy and P_xz swapped": [("q[3] += n[0] * n[1] * wi; q[4] += n[0] * n[2] * wi;",
                               "q[3] += n[0] * n[2] * wi; q[4] += n[0] * n[1] * wi;")],
    "v~ with off-diagonal P": [("double Pd[3] = {Pm[6 * c], Pm[6 * c + 1], Pm[6 * c + 2]};",
                                "double Pd[3] = {Pm[6 * c], Pm[6 * c + 3], Pm[6 * c + 4]};")],
    "J = E instead of E / 4 pi": [("    J[c] = E[c] / (4 * ORC_PI);\n    st[c] = sa[c] + ss[c];",
                                   "    J[c] = E[c];\n    st[c] = sa[c] + ss[c];")],
    # boundary values
    "vacuum zeroes the outgoing rays too": [("  if (!incoming) return val;\n  if (p->bc[d][side] == ORC_VACUUM) return 0.0;",
                                             "  if (p->bc[d][side] == ORC_VACUUM) return 0.0;\n  if (!incoming) return val;")],
    "inflow on the outgoing rays": [("int incoming = side ? (mud < 0) : (mud > 0);",
                                     "int incoming = side ? (mud > 0) : (mud < 0);")],
    "copy from the far end": [("cc[d] = side ? n - 1 : 0;", "cc[d] = side ? 0 : n - 1;")],
    # velocity estimate (sec. 4.5)
    "v~ with -P F": [("double num = rho * v[d] + h * (p->C * rho * v[d] + p->P * F[d]);",
                      "double num = rho * v[d] + h * (p->C * rho * v[d] - p->P * F[d]);")],
    "v~ without P_dd": [("double den = rho + h * (p->C * rho + p->P * (E + Pd[d]) / p->C);",
                         "double den = rho + h * (p->C * rho + p->P * E / p->C);")],
    "v~ over a full step": [("double h = 0.5 * dt * st;", "double h = dt * st;")],
    # absorption, reduced form (sec. 4.3)
    "d_m with +n.v": [("double d = 1.0 + dt * C * sa - dt * sa * vn;", "double d = 1.0 + dt * C * sa + dt * sa * vn;")],
    "e_m without its factor 3": [("double e = dt * sa * (C + 3.0 * vn);", "double e = dt * sa * (C + vn);")],
    "g_m without (n.v)^2": [("double W = p->w[m], g = W * (v2 + vn * vn);", "double W = p->w[m], g = W * v2;")],
    "beta with +v^2/C^2": [("double beta = P * C * (1.0 - v2 / (C * C)) * sa;",
                            "double beta = P * C * (1.0 + v2 / (C * C)) * sa;")],
    "energy row with +S/C": [("(8 * ORC_PI * P * sa * (H0 - S0 / C) - 4 * ORC_PI * beta * J0)",
                              "(8 * ORC_PI * P * sa * (H0 + S0 / C) - 4 * ORC_PI * beta * J0)")],
    "I row with +kappa S": [("I[m] = (r[m] + e * th - kap * S) / d;", "I[m] = (r[m] + e * th + kap * S) / d;")],
    "emission at T^n": [("    if (it == ORC_NEWTON_MAXIT) status = 1;\n    th = pow(T, 4) / (4 * ORC_PI);",
                         "    if (it == ORC_NEWTON_MAXIT) status = 1;\n    th = pow(cs->T0, 4) / (4 * ORC_PI);")],
    # scattering (sec. 4.4)
    "b_l with n.v once": [("*b = -dt * C * ss + 2.0 * dt * ss * vn - dt * ss * v2 / C - dt * ss * vn * vn / C;",
                           "*b = -dt * C * ss + dt * ss * vn - dt * ss * v2 / C - dt * ss * vn * vn / C;")],
    "c_m without its factor 3": [("*c = -3.0 * dt * ss * vn;", "*c = -dt * ss * vn;")],
    "a_m with +n.v": [("*a = (1.0 + dt * C * ss - dt * ss * vn) / p->w[m];", "*a = (1.0 + dt * C * ss + dt * ss * vn) / p->w[m];")],
    # the step: routing of Delta F and the gas sources (sec. 4.1, eqs. momentumchange, kinetichange)
    "Delta F to the smaller opacity": [("int to_scat = ss[c] > sa[c];", "int to_scat = ss[c] < sa[c];")],
    "momentum source without 4 pi": [("double dm = -(4 * ORC_PI * p->P / p->C) * (post[i] - pre[i]);",
                                      "double dm = -(p->P / p->C) * (post[i] - pre[i]);")],
    "momentum source with the wrong sign": [("double dm = -(4 * ORC_PI * p->P / p->C) * (post[i] - pre[i]);",
                                             "double dm = (4 * ORC_PI * p->P / p->C) * (post[i] - pre[i]);")],
    "transport counted as a gas source": [("pre[i] += p->w[m] * p->mu[3 * m + i] * full;",
                                           "pre[i] += p->w[m] * p->mu[3 * m + i] * I0[m];")],
    "gas energy rho R / gamma": [("double kv = rho[c] * p->R / (p->gamma - 1.0);", "double kv = rho[c] * p->R / p->gamma;")],
    "kinetic energy change with the wrong sign": [("dEgas[c] = kv * (T1 - T[c]) + dEK;", "dEgas[c] = kv * (T1 - T[c]) - dEK;")],
    "kinetic energy without the 1/2": [("dEK += ((m0 + dm) * (m0 + dm) - m0 * m0) / (2.0 * rho[c]);",
                                        "dEK += ((m0 + dm) * (m0 + dm) - m0 * m0) / rho[c];")],
    "Newton stopped at 1e-6": [("#define ORC_NEWTON_RTOL 1e-13", "#define ORC_NEWTON_RTOL 1e-6")],
}


def run(name, subs, orig, tmp):
    src = orig
    for old, new in subs:
        if src.count(old) < 1:
            return "not applied: %r not found" % old[:60]
        src = src.replace(old, new)
    path = os.path.join(tmp, "rt_oracle.c")
    with open(path, "w") as f:
        f.write(src)
    lib = os.path.join(tmp, "_liborc_%d.so" % abs(hash(name)))
    env = dict(os.environ, RT_ORACLE_SRC=path, RT_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                       [os.path.join(HERE, t) for t in PINS], cwd=ROOT, env=env, capture_output=True, text=True)
    if r.returncode == 0:
        return "SURVIVED"
    failed = [ln[7:].split(" - ")[0] for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
    return "caught by " + (failed[0] if failed else "an error (rc %d)" % r.returncode)


def main(names):
    with open(SRC) as f:
        orig = f.read()
    todo = {k: v for k, v in MUTATIONS.items() if not names or k in names}
    bad = 0
    with tempfile.TemporaryDirectory() as tmp:
        for name, subs in todo.items():
            verdict = run(name, subs, orig, tmp)
            bad += not verdict.startswith("caught")
            print("%-44s %s" % (name, verdict), flush=True)
    print("%d of %d alterations caught" % (len(todo) - bad, len(todo)))
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
