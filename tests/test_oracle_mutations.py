"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source (a
dropped term, a flipped sign, a wrong factor, a missed mirror), builds it with
gcc, and runs the pin tests against it in a subprocess.  The case passes when
at least one pin fails.  Nothing here touches the GPU or the CUDA library.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "axlbm_oracle.c")

MUTATIONS = {
    "half force dropped from u_z (Eq. 15)":
        ("const double uz = (sz + 0.5 * fext_z) / s0;", "const double uz = sz / s0;"),
    "sign of the radial rate term (Eq. 13)":
        ("(1.0 + over_r(tau * CR[a], r)) / (tau + 0.5)", "(1.0 - over_r(tau * CR[a], r)) / (tau + 0.5)"),
    "mu/r^2 dropped from the u_r denominator (Eq. 16)":
        ("/ (s0 + over_r2(mu0, r));", "/ s0;"),
    "sign in the density (Eq. 17)":
        ("s0 / (1.0 + over_r(0.5 * ur, r))", "s0 / (1.0 - over_r(0.5 * ur, r))"),
    "sign of u_r/r in the source (Eq. 12)":
        ("- over_r(ur, r)) * feq;", "+ over_r(ur, r)) * feq;"),
    "factor 2 in F_r (Eq. 12)":
        ("const double fr = over_r2(-2.0 * mu0", "const double fr = over_r2(-1.0 * mu0"),
    "inertial force dropped (Sec. III C)":
        ("+ over_r(p->rho0 * uth * uth, r);\n    double fz", ";\n    double fz"),
    "second-order equilibrium coefficient (Eq. 6)":
        ("4.5 * eu * eu - 1.5 * usq);\n            const double src",
         "3.0 * eu * eu - 1.5 * usq);\n            const double src"),
    "trapezoidal factor of the source (Eq. 13)":
        ("(1.0 - 0.5 * om) * src;", "src;"),
    "nu/r term of S^g dropped (Eq. 54)":
        ("(2.0 * ur + over_r(nu, r)) * geq", "(2.0 * ur) * geq"),
    "tau_g = tau instead of 2 tau / 3":
        ("const double taug = 2.0 * tau / 3.0;", "const double taug = tau;"),
    "g not odd across the axis":
        ("= s.fr ? -v : v;", "= v;"),
    "moving-wall term doubled":
        ("-v + 0.5 * p->rho0 * wall_uth", "-v + 1.0 * p->rho0 * wall_uth"),
    "temperature source dropped":
        ("const double sh = -over_r(ur, r) * heq;", "const double sh = 0.0 * heq;"),
    "temperature rate without the radial term":
        ("(1.0 + over_r(taut * QR[a], r)) / (taut + 0.5)", "1.0 / (taut + 0.5)"),
    "axis reflection without the r flip":
        ("find9(s.fr ? -CR[a] : CR[a], s.fz ? -CZ[a] : CZ[a])", "find9(CR[a], s.fz ? -CZ[a] : CZ[a])"),
    "mixed top classified by node instead of crossing point":
        ("top_kind_at(p, node_r(p, j) + 0.5 * cr)", "top_kind_at(p, node_r(p, j))"),
    "u_theta not divided by rho0":
        ("        uth /= p->rho0;\n", ""),
    "MRT: momentum correction of Eq. 49 with the wrong sign":
        ("mp[3] -= gamma * ((se / (6.0 * sv)) * e1 + 0.5 * pxx1);", "mp[3] += gamma * ((se / (6.0 * sv)) * e1 + 0.5 * pxx1);"),
    "MRT: correction of Eq. 50 dropped":
        ("    mp[5] -= gamma * pxy1;\n", ""),
    "MRT: source sign of Eq. 51 taken as printed (+)":
        ("src[i] = -over_r(ur, r) * meq[i] + sp[i];", "src[i] = over_r(ur, r) * meq[i] + sp[i];"),
    "MRT: half-source dropped from m^(1)":
        ("const double pxy1 = (m[8] - meq[8]) + 0.5 * src[8];", "const double pxy1 = (m[8] - meq[8]);"),
    "node on the axis: mirror column taken from node 0 instead of node 1":
        ("const size_t x1 = (size_t)k * nr + 1;", "const size_t x1 = (size_t)k * nr + 0;"),
    "node on the axis: 1/r terms not zeroed at r = 0":
        ("return r > 0.0 ? x / r : 0.0;", "return r > 0.0 ? x / r : x / 0.5;"),
    "node on the axis: node 0's outward populations kept":
        ("} else if (p->inner == ORC_AXIS_NODE && s.fr) {\n                    /* leaves through the axis (into the mirror column) */\n                } else {",
         "} else {"),
    "node on the axis: mirror column's g not negated":
        ("if (p->swirl) gn[b * n + y] = -gp[", "if (p->swirl) gn[b * n + y] = gp["),
    "node on the axis: outer wall speed taken at r0 + nr":
        ("(node_r(p, p->nr - 1) + 0.5); /* half-way wall */", "(p->r0 + p->nr);"),
    "wet wall: extrapolated from the wall column itself":
        ("const int jf = on_out ? nr - 2 : j;", "const int jf = on_out ? nr - 1 : j;"),
    "wet wall: wall speed not imposed on g":
        ("const double uth_w = p->omega_w[face] * rb;", "const double uth_w = 0.0;"),
    "wet wall: Dirichlet temperature ignored":
        ("const double t_b = p->t_dirichlet[face] ? p->t_w[face] : temp;", "const double t_b = temp;"),
    "wet wall: equilibrium at the fluid velocity":
        ("const double feq_w = WT[a] * rho_b;", "const double feq_w = feq_f;"),
    "wet wall: non-equilibrium part not relaxed":
        ("f[a * n + xb] = feq_w + (1.0 - om) * (fi[a] - feq_f);", "f[a * n + xb] = feq_w + (fi[a] - feq_f);"),
    "wet wall: density not extrapolated":
        ("const double rho_b = 2.0 * m[0] - m2[0];", "const double rho_b = m[0];"),
    "Zou-He: normal population not bounced back":
        ("        v[3] = v[1];\n", "        v[3] = 0.0;\n"),
    "Zou-He: half-force term missing from the wall velocity":
        ("const double mz = -0.5 * force_at(p, t);", "const double mz = 0.0 * force_at(p, t);"),
    "sign of the buoyancy force":
        ("fz += p->rho0 * p->gbeta * (temp - p->t_ref);", "fz -= p->rho0 * p->gbeta * (temp - p->t_ref);"),
    "lid speed taken at the outer wall instead of at the crossing column":
        ("default: return p->omega_w[face] * node_r(p, j);", "default: return p->omega_w[face] * (p->r0 + p->nr);"),
    "g equilibrium with half its advection term (Eq. 54)":
        ("const double geq = p->rho0 * uth / 4.0 * (1.0 + 2.0 * eu);",
         "const double geq = p->rho0 * uth / 4.0 * (1.0 + 1.0 * eu);"),
    "temperature equilibrium with half its advection term":
        ("const double heq = temp / 4.0 * (1.0 + 2.0 * eu);", "const double heq = temp / 4.0 * (1.0 + 1.0 * eu);"),
    "periodic wrap off by one row":
        ("s.k = ((s.k % p->nz) + p->nz) % p->nz;", "s.k = ((s.k % p->nz) + p->nz - 1) % p->nz;"),
    "MRT: q_x relaxed at the epsilon rate":
        ("    L[4] = sq;\n", "    L[4] = seps;\n"),
    "MRT: p_xy relaxed at the epsilon rate":
        ("    L[8] = sv;\n", "    L[8] = seps;\n"),
    "force taken one step late (after the collision's time)":
        ("return p->az0 * cos(p->omega_t * (double)t);", "return p->az0 * cos(p->omega_t * (double)(t + 1));"),
    "free surface without the flip of e_z":
        ("s.k = s.k < 0 ? -1 - s.k : 2 * p->nz - 1 - s.k;\n            s.fz = 1;",
         "s.k = s.k < 0 ? -1 - s.k : 2 * p->nz - 1 - s.k;\n            s.fz = 0;"),
    "Eq. 57 speed including the azimuthal velocity":
        ("speed[x] = sqrt(m[1] * m[1] + m[2] * m[2]);", "speed[x] = sqrt(m[1] * m[1] + m[2] * m[2] + m[3] * m[3]);"),
    "Eq. 57 speed from the axial velocity alone":
        ("speed[x] = sqrt(m[1] * m[1] + m[2] * m[2]);", "speed[x] = fabs(m[2]);"),
    "Dirichlet temperature wall bounced back with the wrong sign":
        ("p->t_dirichlet[s.face] ? -v + 0.5 * p->t_w[s.face] : v;", "p->t_dirichlet[s.face] ? v + 0.5 * p->t_w[s.face] : v;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mutated = tmp_path / "oracle_mutant.c"
    mutated.write_text(src.replace(old, new, 1))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(lib), str(mutated), "-lm"],
                   check=True)
    env = dict(os.environ, AXLBM_ORACLE_LIB=str(lib))
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                          os.path.join(ROOT, "tests", "test_oracle_mrt.py"),
                          os.path.join(ROOT, "tests", "test_oracle_axis_node.py"),
                          os.path.join(ROOT, "tests", "test_oracle_nee.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"no pin caught: {name}\n{res.stdout[-2000:]}"
