"""Mutation check of the oracle's pins (test infrastructure; not collected by pytest).

Each entry below plants one plausible mistake in the oracle: its BSSN right-hand side,
constraints, stencils, boundary condition, det enforcement or integrators: a wrong coefficient, sign, index or a dropped term. For every
mutant the script runs the oracle pin tests on a copy of the repository and reports
whether some pin fails ("killed") or all pass ("SURVIVED").

    python tests/mutants/run_oracle_mutants.py SCRATCH_DIR [name filter ...]

SCRATCH_DIR receives a copy of oracle/, tests/ and the package's Python files. The
repository itself is never modified.
"""
import os
import shutil
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

MUT = [
 ("eps: 2/3 trace term", "t += (2.0 / 3.0) * G.gb[i][j] * (al * G.trA - divbar);", "t += (1.0 / 3.0) * G.gb[i][j] * (al * G.trA - divbar);"),
 ("eps: -2 alpha A", "t -= 2.0 * al * F->A[i][j];", "t -= al * F->A[i][j];"),
 ("eps: Lie second term", "for (int k = 0; k < 3; k++) t += F->eps[k][j] * F->dbeta[k][i] + F->eps[i][k] * F->dbeta[k][j];", "for (int k = 0; k < 3; k++) t += F->eps[k][j] * F->dbeta[k][i];"),
 ("eps: Db term", "for (int k = 0; k < 3; k++) t += M->g[j][k] * Db[k][i] + M->g[i][k] * Db[k][j];", "for (int k = 0; k < 3; k++) t += M->g[j][k] * Db[k][i] + M->g[i][k] * Db[j][k];"),
 ("X: 4 alpha dphi dphi", "4.0 * al * G.dphi[i] * G.dphi[j]", "2.0 * al * G.dphi[i] * G.dphi[j]"),
 ("X: 2 dalpha dphi", "2.0 * (F->dalpha[i] * G.dphi[j] + F->dalpha[j] * G.dphi[i])", "1.0 * (F->dalpha[i] * G.dphi[j] + F->dalpha[j] * G.dphi[i])"),
 ("X: -DDal sign", "- DDal[i][j] + al * G.Ric[i][j];", "+ DDal[i][j] + al * G.Ric[i][j];"),
 ("X: -2 alpha DDphi", "X[i][j] = -2.0 * al * G.DDphi[i][j]", "X[i][j] = -1.0 * al * G.DDphi[i][j]"),
 ("A: 2/3 A divbar", "t -= (2.0 / 3.0) * F->A[i][j] * divbar;", "t -= (1.0 / 3.0) * F->A[i][j] * divbar;"),
 ("A: -2 alpha AA", "t -= 2.0 * al * AA_ij;", "t -= al * AA_ij;"),
 ("A: + alpha A K", "t += al * F->A[i][j] * K;", "t -= al * F->A[i][j] * K;"),
 ("A: trace-free 1/3", "t += W2 * (X[i][j] - (1.0 / 3.0) * G.gb[i][j] * trX);", "t += W2 * (X[i][j] - 0.5 * G.gb[i][j] * trX);"),
 ("A: Lie second term", "for (int k = 0; k < 3; k++) t += F->A[k][j] * F->dbeta[k][i] + F->A[i][k] * F->dbeta[k][j];", "for (int k = 0; k < 3; k++) t += F->A[k][j] * F->dbeta[k][i];"),
 ("W: sign of alpha K", "(1.0 / 3.0) * W * (divbar - al * K)", "(1.0 / 3.0) * W * (divbar + al * K)"),
 ("K: K^2/3", "(1.0 / 3.0) * al * K * K", "0.5 * al * K * K"),
 ("K: alpha AA", "+ al * G.AA - W2", "+ 2.0 * al * G.AA - W2"),
 ("K: 2 grad alpha grad phi", "(lapl_al + 2.0 * grad_ap)", "(lapl_al + grad_ap)"),
 ("Lam: 2/3 Delta divbar", "t += (2.0 / 3.0) * G.Dvec[i] * divbar;", "t += (1.0 / 3.0) * G.Dvec[i] * divbar;"),
 ("Lam: 1/3 grad divbar", "t += (1.0 / 3.0) * G.gbinv[i][k] * d_divbar[k];", "t += (2.0 / 3.0) * G.gbinv[i][k] * d_divbar[k];"),
 ("Lam: 6 alpha dphi", "(F->dalpha[j] - 6.0 * al * G.dphi[j])", "(F->dalpha[j] - 4.0 * al * G.dphi[j])"),
 ("Lam: 2 alpha A Delta", "t += 2.0 * al * G.Auu[j][k] * G.Dup[i][j][k];", "t += al * G.Auu[j][k] * G.Dup[i][j][k];"),
 ("Lam: 4/3 alpha dK", "t -= (4.0 / 3.0) * al * G.gbinv[i][j] * F->dK[j];", "t -= (2.0 / 3.0) * al * G.gbinv[i][j] * F->dK[j];"),
 ("Lam: Lie sign", "lie -= F->Lam[j] * F->dbeta[i][j];", "lie += F->Lam[j] * F->dbeta[i][j];"),
 ("Lam: LapB", "for (int k = 0; k < 3; k++) t += G.gbinv[j][k] * DDb[i][j][k];", "for (int k = 0; k < 3; k++) t += G.gbinv[j][k] * DDb[i][k][k];"),
 ("alpha: 1+log 2", "double r_al = -2.0 * al * K + F->adv_alpha;", "double r_al = -al * K + F->adv_alpha;"),
 ("beta: B coefficient", "r_beta[i] = F->B[i] + F->adv_beta[i];", "r_beta[i] = 0.5 * F->B[i] + F->adv_beta[i];"),
 ("B: eta sign", "- p->eta * F->B[i] + F->adv_B[i];", "+ p->eta * F->B[i] + F->adv_B[i];"),
 ("Ric: -1/2 r1", "G->Ric[i][j] = -0.5 * r1 + 0.5 * r2 + r3 + r4;", "G->Ric[i][j] = -0.25 * r1 + 0.5 * r2 + r3 + r4;"),
 ("Ric: r2", "G->Ric[i][j] = -0.5 * r1 + 0.5 * r2 + r3 + r4;", "G->Ric[i][j] = -0.5 * r1 + r2 + r3 + r4;"),
 ("Ric: r3 sign", "G->Ric[i][j] = -0.5 * r1 + 0.5 * r2 + r3 + r4;", "G->Ric[i][j] = -0.5 * r1 + 0.5 * r2 - r3 + r4;"),
 ("Ric: r4 third term", "G->Dup[m][k][j] * G->Dl[i][m][l] +\n                             G->Dup[m][i][k] * G->Dl[m][j][l];", "G->Dup[m][k][j] * G->Dl[i][m][l];"),
 ("Ric: r4 first index", "s += G->Dup[m][k][i] * G->Dl[j][m][l]", "s += G->Dup[m][k][i] * G->Dl[m][j][l]"),
 ("H: 2/3 K^2", "H[idx] = (2.0 / 3.0) * F.K * F.K - G.AA", "H[idx] = (1.0 / 3.0) * F.K * F.K - G.AA"),
 ("H: AA sign", "H[idx] = (2.0 / 3.0) * F.K * F.K - G.AA", "H[idx] = (2.0 / 3.0) * F.K * F.K + G.AA"),
 ("H: 8 gp", "(Rs - 8.0 * gp - 8.0 * lp)", "(Rs - 4.0 * gp - 8.0 * lp)"),
 ("H: 8 lp", "(Rs - 8.0 * gp - 8.0 * lp)", "(Rs - 8.0 * gp - 4.0 * lp)"),
 ("M: 6 Abar dphi", "(div + dterm + 6.0 * ph - (2.0 / 3.0) * kk)", "(div + dterm + 4.0 * ph - (2.0 / 3.0) * kk)"),
 ("M: 2/3 dK", "(div + dterm + 6.0 * ph - (2.0 / 3.0) * kk)", "(div + dterm + 6.0 * ph - (1.0 / 3.0) * kk)"),
 ("M: Delta term sign", "(div + dterm + 6.0 * ph", "(div - dterm + 6.0 * ph"),
 ("KO: 1/64 normalisation", "ko += p->ko_sigma[gf] / (64.0 * h[d] * R.S[d]) * orc_ko6(f, st[d]);", "ko += p->ko_sigma[gf] / (32.0 * h[d] * R.S[d]) * orc_ko6(f, st[d]);"),
 ("upwind: direction", "fwd[k] = vet > 0.0;", "fwd[k] = vet < 0.0;"),
 ("outer BC: 1/r term", "rhs[gf * T + idx] = -p->wavespeed[gf] * (radial + (f[0] - p->f_inf[gf]) / r);", "rhs[gf * T + idx] = -p->wavespeed[gf] * radial;"),
 ("outer BC: sign", "rhs[gf * T + idx] = -p->wavespeed[gf] * (radial + (f[0] - p->f_inf[gf]) / r);", "rhs[gf * T + idx] = p->wavespeed[gf] * (radial + (f[0] - p->f_inf[gf]) / r);"),
 ("RK4: weight of k2", "(k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i])", "(k1[i] + k2[i] + 3.0 * k3[i] + k4[i])"),
 ("RK4: midpoint", "yt[i] = y[i] + dt * k3[i];", "yt[i] = y[i] + 0.5 * dt * k3[i];"),
 ("det: exponent", "double f1 = expm1(-log1p(e1 + e2 + e3) / 3.0);", "double f1 = expm1(-log1p(e1 + e2 + e3) / 2.0);"),
 ("SSPRK3: stage 2", "y2[i] = 0.75 * y[i] + 0.25 * (y1[i] + dt * k[i]);", "y2[i] = 0.5 * y[i] + 0.5 * (y1[i] + dt * k[i]);"),
 ("psi4: E kk sign", "E[i][j] = Ric[i][j] - kk + F->K * Kd[i][j];", "E[i][j] = Ric[i][j] + kk + F->K * Kd[i][j];"),
 ("psi4: E K Kd", "E[i][j] = Ric[i][j] - kk + F->K * Kd[i][j];", "E[i][j] = Ric[i][j] - kk;"),
 ("psi4: B derivative index", "if (e) b += gam[i][m] * e * DK[k][l][j];", "if (e) b += gam[i][m] * e * DK[l][k][j];"),
 ("psi4: real part B sign", "psi4[idx] = -0.5 * (Et[1][1] - Et[2][2]) + Bt[1][2];", "psi4[idx] = -0.5 * (Et[1][1] - Et[2][2]) - Bt[1][2];"),
 ("psi4: imaginary part E", "psi4[T + idx] = Et[1][2] + 0.5 * (Bt[1][1] - Bt[2][2]);", "psi4[T + idx] = -Et[1][2] + 0.5 * (Bt[1][1] - Bt[2][2]);"),
 ("psi4: Gram-Schmidt step", "for (int d = 0; d < 3; d++) u[a][d] -= dot * u[b][d];", "for (int d = 0; d < 3; d++) u[a][d] -= 0.0 * dot * u[b][d];"),
 ("parity: tensor sign", "for (int s = 0; s < 6; s++) par[4 + s] = (int8_t)(pd[SYM_I[s]] * pd[SYM_J[s]]);", "for (int s = 0; s < 6; s++) par[4 + s] = (int8_t)(pd[SYM_I[s]]);"),
 ("rescale: vector dS sign", "Rd[k] = -R->dS[i][k] / (S * S);", "Rd[k] = R->dS[i][k] / (S * S);"),
 ("rescale: vector ddS cross term", "+ 2.0 * R->dS[i][k] * R->dS[i][l] / (S * S * S);", "+ R->dS[i][k] * R->dS[i][l] / (S * S * S);"),
 ("rescale: tensor cross term", "+ R->dS[i][k] * R->dS[j][l] + R->dS[i][l] * R->dS[j][k] +", "+ 2.0 * R->dS[i][k] * R->dS[j][l] +"),
 ("BL: psi", "psi += mass[q] / (2.0 * d);", "psi += mass[q] / d;"),
 ("ord8: KO normalisation", "ko += p->ko_sigma[gf] / (ldexp(1.0, 2 * r) * h[d] * R.S[d]) * sten(f, st[d], Wd.ko, -r, r);", "ko += p->ko_sigma[gf] / (ldexp(1.0, 2 * r - 1) * h[d] * R.S[d]) * sten(f, st[d], Wd.ko, -r, r);"),
 ("ord8: upwind window", "for (int i = 0; i < n; i++) x[i] = i - (m - 1);", "for (int i = 0; i < n; i++) x[i] = i - (m + 1);"),
 ("SSPRK3: stage 3", "y[i] = (1.0 / 3.0) * y[i] + (2.0 / 3.0) * (y2[i] + dt * k[i]);", "y[i] = 0.5 * y[i] + 0.5 * (y2[i] + dt * k[i]);"),
 ("Ric: DLam Gamma sign", "for (int m = 0; m < 3; m++) s += M->Gam[k][j][m] * F->Lam[m];", "for (int m = 0; m < 3; m++) s -= M->Gam[k][j][m] * F->Lam[m];"),
 ("DDphi: dW dW sign", "+ F->dW[i] * F->dW[j] / (2.0 * F->W * F->W);", "- F->dW[i] * F->dW[j] / (2.0 * F->W * F->W);"),
 ("DDphi: connection sign", "for (int k = 0; k < 3; k++) s -= G->Gb[k][i][j] * G->dphi[k];", "for (int k = 0; k < 3; k++) s += G->Gb[k][i][j] * G->dphi[k];"),
 ("DDal: connection sign", "for (int k = 0; k < 3; k++) s -= G.Gb[k][i][j] * F->dalpha[k];", "for (int k = 0; k < 3; k++) s += G.Gb[k][i][j] * F->dalpha[k];"),
 ("Dtr: 1/2", "Dtr[m] = 0.5 * s;", "Dtr[m] = s;"),
 ("divbar: Dtr beta sign", "for (int m = 0; m < 3; m++) divbar += Dtr[m] * F->beta[m];", "for (int m = 0; m < 3; m++) divbar -= Dtr[m] * F->beta[m];"),
 ("DDb: second connection sign", "s += M->Gam[i][l][m] * Db[m][k] - M->Gam[m][l][k] * Db[i][m];", "s += M->Gam[i][l][m] * Db[m][k] + M->Gam[m][l][k] * Db[i][m];"),
]

TESTS = ["tests/test_oracle_grid.py", "tests/test_oracle_stencils.py", "tests/test_oracle_upwind.py", "tests/test_oracle_order8.py", "tests/test_oracle_momentum.py",
         "tests/test_oracle_physics.py", "tests/test_oracle_gauge.py", "tests/test_oracle_lambda_pin.py",
         "tests/test_oracle_kerr_schild.py", "tests/test_oracle_psi4.py"]


def main():
    if len(sys.argv) < 2:
        sys.exit(__doc__)
    work = os.path.abspath(sys.argv[1])
    only = sys.argv[2:]
    if work == ROOT:
        sys.exit("SCRATCH_DIR must not be the repository itself")
    for d in ("oracle", "tests", "paper_2505_00097_gb300"):
        shutil.rmtree(os.path.join(work, d), ignore_errors=True)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(work, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(work, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    pkg = os.path.join(work, "paper_2505_00097_gb300")
    os.makedirs(pkg)
    for f in os.listdir(os.path.join(ROOT, "paper_2505_00097_gb300")):
        if f.endswith(".py"):
            shutil.copy(os.path.join(ROOT, "paper_2505_00097_gb300", f), pkg)
    src = os.path.join(work, "oracle", "nr_oracle.c")
    orig = open(src).read()
    survivors = []
    for name, old, new in MUT:
        if only and not any(o in name for o in only):
            continue
        assert orig.count(old) == 1, (name, orig.count(old))
        open(src, "w").write(orig.replace(old, new))
        t0 = time.time()
        r = subprocess.run([sys.executable, "-m", "pytest", *TESTS, "-x", "-q", "-p", "no:cacheprovider"],
                           cwd=work, capture_output=True, text=True)
        first = next((ln.split("::")[-1][:70] for ln in r.stdout.splitlines() if ln.startswith("FAILED")), "")
        killed = r.returncode != 0
        print(f"{'killed  ' if killed else 'SURVIVED'} {time.time() - t0:5.1f}s  {name:32s} {first}", flush=True)
        if not killed:
            survivors.append(name)
    open(src, "w").write(orig)
    print("survivors:", survivors)
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main())
