"""Planted mistakes: the pins pin the oracle.

Each case copies the oracle's C sources, plants one plausible mistake in the
copy (a flipped sign, a dropped term, a wrong index or coefficient), builds it,
and runs every oracle pin against it (tests/test_oracle_*.py, through the
oracle's HGKS_ORACLE_LIB hook). At least one pin must fail for every case: a
mistake of that kind anywhere in the oracle would not go unnoticed. The copies
are built in a temporary directory; the oracle itself is not touched."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys
import tempfile

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join(ROOT, "tests", f)
        for f in ("test_oracle_pins.py", "test_oracle_fd.py", "test_oracle_force.py", "test_oracle_hex.py")]

# (what the mistake is, file, text as written, text with the mistake)
PLANTED = [
    # Maxwellian moments (Sec. 2)
    ("half-range <u>: sign of the Gaussian term", "orc_gks.c",
     "mu[1] = U * mu[0] + ex;", "mu[1] = U * mu[0] - ex;"),
    ("moment recursion: k instead of k + 1", "orc_gks.c",
     "mu[n + 2] = U * mu[n + 1] + (n + 1) / (2.0 * lam) * mu[n];", "mu[n + 2] = U * mu[n + 1] + n / (2.0 * lam) * mu[n];"),
    ("<xi^4> without the 2K term", "orc_gks.c", "mxi[2] = (K * K + 2.0 * K)", "mxi[2] = (K * K + K)"),
    # time evolution and flux (Eq. (flux), Sec. 4.1, Sec. 5)
    ("collision time without the pressure jump", "orc_gks.c",
     "p->tau_eps * dt + p->tau_C * jump * dt", "p->tau_eps * dt"),
    ("viscous collision time with the left pressure instead of Q0's", "orc_gks.c",
     "p->viscous ? p->mu / pp0", "p->viscous ? p->mu / prl"),
    ("time coefficient c2: sign of tau dt (1 + e)", "orc_gks.c",
     "- tau * dt * (1.0 + e);", "+ tau * dt * (1.0 + e);"),
    ("time coefficient c3: sign of tau dt", "orc_gks.c",
     "double c3 = 0.5 * dt * dt - tau * dt", "double c3 = 0.5 * dt * dt + tau * dt"),
    ("time coefficient c5: e dropped", "orc_gks.c", "- tau * dt * e;", "- tau * dt;"),
    ("time slope A: compatibility sign", "orc_gks.c",
     "for (int i = 0; i < 5; i++) rhs[i] = -rhs[i];", "for (int i = 0; i < 5; i++) rhs[i] = 2.0 * rhs[i];"),
    ("Q0 from the full-range right Maxwellian", "orc_gks.c",
     "Q0[a] = p_int(&ps, &Tlp) + p_int(&ps, &Trm);", "Q0[a] = p_int(&ps, &Tlp) + p_int(&ps, &Tr);"),
    ("equilibrium slopes from the left gradient only", "orc_gks.c",
     "dQ0[c] = 0.5 * (dWl[5 * d + c] + dWr[5 * d + c]);", "dQ0[c] = dWl[5 * d + c];"),
    ("flux: tau c4 A term of the left side dropped", "orc_gks.c",
     "+ c4 * fl[a] - c5 * fal[a] - tau * c4 * fAl[a]", "+ c4 * fl[a] - c5 * fal[a]"),
    ("Prandtl fix: factor Pr - 1 instead of 1/Pr - 1", "orc_gks.c",
     "F[4] += (1.0 / p->Pr - 1.0) * q;", "F[4] += (p->Pr - 1.0) * q;"),
    ("point value: sign of the tau abar term", "orc_gks.c",
     "((ts + tau) * es - tau) * mab[a]", "((ts + tau) * es + tau) * mab[a]"),
    ("point value: t* term of the left side dropped", "orc_gks.c",
     "+ es * (ml[a] - (tau + ts) * mal[a] - tau * mAl[a])", "+ es * (ml[a] - tau * mal[a] - tau * mAl[a])"),
    # boundary images (Sec. 5.1, 5.2)
    ("far field: free stream rotated by the transposed face frame", "orc_gks.c",
     "u[i] = T3[3 * i] * p->u_inf[0] + T3[3 * i + 1] * p->u_inf[1] + T3[3 * i + 2] * p->u_inf[2];",
     "u[i] = T3[i] * p->u_inf[0] + T3[i + 3] * p->u_inf[1] + T3[i + 6] * p->u_inf[2];"),
    ("moving wall: image velocity u_w - u instead of 2 u_w - u", "orc_gks.c",
     "ug[i] = vel_odd[i] ? 2.0 * uw[i] - u[i] : u[i];", "ug[i] = vel_odd[i] ? uw[i] - u[i] : u[i];"),
    ("slip wall reflects a tangential velocity", "orc_gks.c",
     "if (tag == 3) { vel_odd[0] = 1; vel_odd[1] = 0; vel_odd[2] = 0; }",
     "if (tag == 3) { vel_odd[0] = 1; vel_odd[1] = 1; vel_odd[2] = 0; }"),
    ("isothermal wall does not reflect the temperature", "orc_gks.c",
     "T_odd = (tag == 1 || tag == 2)", "T_odd = (tag == 2)"),
    ("wall image keeps the normal derivatives", "orc_gks.c",
     "double sn = d == 0 ? -1.0 : 1.0;", "double sn = 1.0;"),
    ("far field from the interior density", "orc_gks.c",
     "Wr[0] = r; Wr[1] = r * u[0]; Wr[2] = r * u[1]; Wr[3] = r * u[2];",
     "r = Wl[0]; Wr[0] = r; Wr[1] = r * u[0]; Wr[2] = r * u[1]; Wr[3] = r * u[2];"),
    ("isothermal image keeps the cell's density ratio p/T_g (mass leaks through the wall)", "orc_gks.c",
     "rg = rho * Ml / Mg;", "rg = pr / Tg;"),
    ("isothermal image density from the wall temperature's mean speed only", "orc_gks.c",
     "Mg = 0.5 * Un * erfc(-sqrt(lam_g) * Un)", "Mg = 0.5 * Un * erfc(-sqrt(lam_l) * Un)"),
    ("wall faces carry mass", "orc_solver.c",
     "if (Rr < 0 && m->ftag[f] >= 1 && m->ftag[f] <= 4) Fg[0] = 0.0;", "if (Rr < 0 && m->ftag[f] >= 1 && m->ftag[f] <= 3) Fg[0] = 0.0;"),
    ("time slope of g0 from the left state", "orc_gks.c",
     "time_slope(p0, K, ab, Ab);", "time_slope(pl, K, ab, Ab);"),
    # reconstruction (Sec. 3, Eq. (weno), characteristic variables of Sec. 5)
    ("eigenvector u + a with H - u a", "orc_recon.c",
     "{1, u + a, v, w, H + u * a}", "{1, u + a, v, w, H - u * a}"),
    ("characteristic projection at the left state, not the face average", "orc_recon.c",
     "Qs[c] = R_ >= 0 ? 0.5 * (Q[5 * L_ + c] + Q[5 * R_ + c]) : Q[5 * i + c];",
     "Qs[c] = Q[5 * L_ + c];"),
    ("Gauss-point gradient not rescaled by h", "orc_recon.c",
     "qg[j][c] = grad[j] / m->h[i];", "qg[j][c] = grad[j];"),
    ("Eq. (weno): gamma_m / gamma_0 taken as gamma_m", "orc_recon.c",
     "val -= gam_m / g0eff * Pm_[mm];", "val -= gam_m * Pm_[mm];"),
    ("beta_0 without its second-derivative term", "orc_recon.c",
     "s += hxx * hxx + hyy * hyy + hzz * hzz", "s += 0.0 * hxx * hxx + hyy * hyy + hzz * hzz"),
    ("tau_Z without the 1/M", "orc_recon.c",
     "tz += fabs(beta[0] - beta[1 + mm]) / M;", "tz += fabs(beta[0] - beta[1 + mm]);"),
    ("nonlinear weight of P0 with beta_1", "orc_recon.c",
     "om[0] = gam0 * (1.0 + tz / (beta[0] + p->weno_eps));", "om[0] = gam0 * (1.0 + tz / (beta[1] + p->weno_eps));"),
    # compact HWENO (Sec. 3.3, Eq. (compact-big-1/2), Eq. (derivative))
    ("HWENO: neighbour gradients taken from the target", "orc_recon.c",
     "for (int j = 0; j < 3; j++) data[nfc + 3 * k + j] = G[15 * ck + 3 * c + j];",
     "for (int j = 0; j < 3; j++) data[nfc + 3 * k + j] = G[15 * i + 3 * c + j];"),
    ("HWENO sub-stencil: the neighbour's gradient dropped", "orc_recon.c",
     "if (jm >= 0) for (int j = 0; j < 3; j++) dm[4 + j] = G[15 * jm + 3 * c + j];", ""),
    ("singular quadratic fits: the stencil stops growing at 12 cells", "orc_mesh.c",
     "const int cap = hex ? 24 : 16;", "const int cap = 12;"),
    ("HWENO fit: equality rows without the target's own average", "orc_mesh.c",
     "for (int d = 0; d < 9; d++) C[r][d] = av[d] - avg_i[d];", "for (int d = 0; d < 9; d++) C[r][d] = av[d];"),
    ("HWENO fit: gradient data not scaled by h", "orc_mesh.c",
     "double dval = m->h[rk->cell];", "double dval = 1.0;"),
    ("HWENO sub-stencil fit: gradient data not scaled by h", "orc_mesh.c",
     "rhs[j] = (hk[k] / m->h[i]) * hk[k];", "rhs[j] = hk[k] / m->h[i];"),
    ("HWENO fit: gradient rows and data without the h_k weights", "orc_mesh.c",
     ("B[3 * k + j][d] = (hk / m->h[i]) * av[d];", "double dval = m->h[rk->cell];"),
     ("B[3 * k + j][d] = av[d];", "double dval = m->h[i];")),
    ("WENO big-stencil fit weighted (rows and data) instead of plain least squares", "orc_mesh.c",
     ("for (int d = 0; d < 9; d++) A[r * 9 + d] = av[d] - avg_i[d];",
      "for (int d = 0; d < 9; d++) for (int r = 0; r < F->n_big; r++) F->X0[d][r] = X[d * F->n_big + r];"),
     ("for (int d = 0; d < 9; d++) A[r * 9 + d] = (1.0 + 0.5 * r) * (av[d] - avg_i[d]);",
      "for (int d = 0; d < 9; d++) for (int r = 0; r < F->n_big; r++) F->X0[d][r] = (1.0 + 0.5 * r) * X[d * F->n_big + r];")),
    ("compact gradient not divided by the volume", "orc_solver.c",
     "if (Gnew) for (int64_t i = 0; i < nc; i++) for (int c = 0; c < 15; c++) Gnew[15 * i + c] /= m->vol[i];", ""),
    ("compact gradient from the face flux instead of the point value", "orc_solver.c",
     "Gnew[15 * L + 3 * c + d] += Pf[5 * f + c] * n[d];", "Gnew[15 * L + 3 * c + d] += Ff[5 * f + c] * n[d];"),
    ("point value at t = 0 regardless of the reading", "orc_gks.c",
     "double ts = p->tstar_end ? dt : 0.0", "double ts = 0.0"),
    # geometry and fits (Sec. 2, Sec. 3.1 - 3.3)
    ("face Gauss points at (1/2, 1/4, 1/4)", "orc_mesh.c",
     "(2.0 / 3.0) * vv[g][d] + (1.0 / 6.0) *", "(1.0 / 2.0) * vv[g][d] + (1.0 / 4.0) *"),
    ("tetrahedron rule collapsed to the centroid", "orc_mesh.c",
     "QA = 0.5854101966249685, QB = 0.1381966011250105;", "QA = 0.25, QB = 0.25;"),
    ("big-stencil rows without the target's own average", "orc_mesh.c",
     "for (int d = 0; d < 9; d++) A[r * 9 + d] = av[d] - avg_i[d];", "for (int d = 0; d < 9; d++) A[r * 9 + d] = av[d];"),
    ("tetrahedron volume / 3", "orc_mesh.c",
     "e1[2] * c[2]) / 6.0;", "e1[2] * c[2]) / 3.0;"),
    ("sub-stencil 4 paired with the wrong triple", "orc_mesh.c",
     "{{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {2, 0, 3}}", "{{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {2, 0, 1}}"),
    ("sub-stencil without the neighbours of neighbour m", "orc_mesh.c",
     "for (int q = 0; q < 4; q++) { double s[3]; int64_t k = nb_of(m, &rm, q, s); add_ref(F->sub[mm], &F->n_sub[mm], ORC_MAXSUB, i, k, s); }",
     "for (int q = 0; q < 1; q++) { double s[3]; int64_t k = nb_of(m, &rm, q, s); add_ref(F->sub[mm], &F->n_sub[mm], ORC_MAXSUB, i, k, s); }"),
    # hexahedral cells (Sec. 3.1)
    ("hexahedron: a sub-stencil across an edge instead of a corner", "orc_mesh.c",
     "{5, 3, 4}, {5, 4, 1}}", "{5, 3, 4}, {5, 4, 2}}"),
    ("hexahedron: sub-stencils of the face-0 corners only", "orc_mesh.c",
     "const int nsub = hex ? 8 : 4;", "const int nsub = hex ? 4 : 4;"),
    ("hexahedron: big stencil from four of the six faces", "orc_mesh.c",
     "for (int q = 0; q < nfc; q++) { double s[3]; int64_t k = nb_of(m, l1 + a, q, s);",
     "for (int q = 0; q < 4; q++) { double s[3]; int64_t k = nb_of(m, l1 + a, q, s);"),
    ("hexahedron: Gauss points of the quadrilateral at 1/2 -+ 1/(2 sqrt 2)", "orc_mesh.c",
     "gl = 0.5 - 0.5 / sqrt(3.0), gh = 0.5 + 0.5 / sqrt(3.0);", "gl = 0.5 - 0.5 / sqrt(2.0), gh = 0.5 + 0.5 / sqrt(2.0);"),
    ("hexahedron: equal Gauss weights on a quadrilateral", "orc_mesh.c",
     "m->fgw[4 * f + g] = jac[g] / jsum;", "m->fgw[4 * f + g] = 0.25;"),
    ("hexahedron: face area from one triangle of the quadrilateral", "orc_mesh.c",
     "for (int d = 0; d < 3; d++) { d1[d] = c[d] - a[d]; d2[d] = e[d] - b[d];",
     "for (int d = 0; d < 3; d++) { d1[d] = c[d] - a[d]; d2[d] = e[d] - a[d];"),
    ("hexahedron: centroid = mean of the vertices", "orc_mesh.c",
     "for (int d = 0; d < 3; d++) m->cen[3 * i + d] = cx[d] / vol;",
     "for (int d = 0; d < 3; d++) { m->cen[3 * i + d] = 0.0; for (int a = 0; a < 8; a++) m->cen[3 * i + d] += 0.125 * xyz[3 * cells[8 * i + a] + d]; }"),
    ("hexahedron: 4-point rule with a wrong outer node", "orc_mesh.c",
     "b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));", "b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(5.0 / 6.0));"),
    ("hexahedron: Jacobian determinant with a wrong cofactor sign", "orc_mesh.c",
     "J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +", "J[0][1] * (J[1][0] * J[2][2] + J[1][2] * J[2][0]) +"),
    ("quadrilateral faces weighted 1/3 like triangles", "orc_solver.c",
     "const double wS = m->farea[f] * m->fgw[ngp * f + g];", "const double wS = m->farea[f] / 3.0;"),
    ("hexahedron: compact fit without the gradients of the last two neighbours", "orc_mesh.c",
     "for (int col = 0; col < nfc + 3 * (1 + nfc); col++) {", "for (int col = 0; col < nfc + 3 * (1 + nfc) - 6; col++) {"),
    # dense linear algebra (the library primitives the oracle's steps call)
    ("elimination without pivoting", "orc_linalg.c",
     "if (fabs(M[r * (n + 1) + c]) > best) { best = fabs(M[r * (n + 1) + c]); piv = r; }",
     "if (0) { best = fabs(M[r * (n + 1) + c]); piv = r; }"),
    ("back substitution skips the last column", "orc_linalg.c",
     "for (int j = i + 1; j < n; j++) s -= M[i * (n + 1) + j] * x[j];",
     "for (int j = i + 1; j < n - 1; j++) s -= M[i * (n + 1) + j] * x[j];"),
    # residual, implicit system, solver (Eq. (finite), (derivative), (deri-matrix), (precond), Algorithm 1)
    ("local time step without the sound speed", "orc_solver.c",
     "pr[3] * n[2]) + a + nu);", "pr[3] * n[2]) + nu);"),
    ("flux added with the wrong sign on the right cell", "orc_solver.c",
     "if (Rr >= 0) R[5 * Rr + c] += Ff[5 * f + c];", "if (Rr >= 0) R[5 * Rr + c] -= Ff[5 * f + c];"),
    ("compact gradient: wrong sign on the right cell", "orc_solver.c",
     "if (Rr >= 0) Gnew[15 * Rr + 3 * c + d] -= Pf[5 * f + c] * n[d];",
     "if (Rr >= 0) Gnew[15 * Rr + 3 * c + d] += Pf[5 * f + c] * n[d];"),
    ("A without |Omega| / dt", "orc_solver.c",
     "D[k] = (k % 6 == 0) ? m->vol[i] / dt[i] : 0.0;", "D[k] = (k % 6 == 0) ? 0.5 * m->vol[i] / dt[i] : 0.0;"),
    ("A: sign of lambda in the diagonal block", "orc_solver.c",
     "D[k] += 0.5 * (J[k] + (k % 6 == 0 ? lam : 0.0)) * S;", "D[k] += 0.5 * (J[k] - (k % 6 == 0 ? lam : 0.0)) * S;"),
    ("A: off-diagonal block with the row cell's Jacobian", "orc_solver.c",
     "orc_euler_jacobian(Q + 5 * j, n, p->gamma, J);", "orc_euler_jacobian(Q + 5 * i, n, p->gamma, J);"),
    ("Jacobi sweep adds the off-diagonal product", "orc_solver.c",
     "s -= off[25 * m->nfc * i + 25 * q + 5 * r + c] * prev[5 * j + c];",
     "s += off[25 * m->nfc * i + 25 * q + 5 * r + c] * prev[5 * j + c];"),
    ("Givens rotation: sign of s", "orc_solver.c",
     "H[(j + 1) * mk + k] = -s * h1 + c * h2;", "H[(j + 1) * mk + k] = s * h1 + c * h2;"),
    ("back substitution adds", "orc_solver.c", "s -= H[j * mk + k] * y[k];", "s += H[j * mk + k] * y[k];"),
    ("the steady loop takes a zero reference as a drop", "orc_solver.c",
     "if (res0 > 0.0 && res <= drop * res0)", "if (res <= drop * res0)"),
    ("density residual norm without the volume", "orc_solver.c",
     "s += fabs(R[5 * i]) / m->vol[i];", "s += fabs(R[5 * i]);"),
    ("matrix-free product: sign of the Frechet difference", "orc_solver.c",
     "y[k] = m->vol[i] / dt[i] * x[k] - (Ls[k] - LQ[k]) / sigma;", "y[k] = m->vol[i] / dt[i] * x[k] + (Ls[k] - LQ[k]) / sigma;"),
]


def _run_case(case, workdir):
    name, fname, orig, planted = case
    d = tempfile.mkdtemp(dir=workdir)
    for f in O.SOURCES + ["orc.h"]:
        shutil.copy(os.path.join(O.HERE, f), d)
    path = os.path.join(d, fname)
    src = open(path).read()
    for o, pl in zip(*((orig, planted) if isinstance(orig, tuple) else ((orig,), (planted,)))):
        assert src.count(o) == 1, f"{name}: the text to change occurs {src.count(o)} times in {fname}"
        src = src.replace(o, pl)
    open(path, "w").write(src)
    lib = O.compile_library(d, os.path.join(d, "liboracle_planted.so"))
    env = dict(os.environ, HGKS_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "not gpu", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    failed = sorted(set(re.findall(r"^FAILED (\S+?)(?:\[| - |$)", r.stdout, flags=re.M)))
    return name, r.returncode, failed, r.stdout[-2000:]


def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as work:
        with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
            results = list(ex.map(lambda c: _run_case(c, work), PLANTED))
    survived = [(n, rc, tail) for n, rc, failed, tail in results if rc != 1 or not failed]
    for n, rc, failed, _ in results:
        print(f"{n}: caught by {', '.join(f.split('::')[-1] for f in failed) or '-'}")
    assert not survived, "planted mistakes no pin caught: " + "; ".join(f"{n} (pytest exit {rc})" for n, rc, _ in survived)
