"""Mutation check of the CPU test of the kernels' arithmetic (test infrastructure; not
collected by pytest).

Each entry below plants one mistake in a copy of the per-point CUDA header
(csrc/bssn_point.cuh): a wrong coefficient or sign, a dropped term, a structural-zero
predicate that skips a term which is not zero, a lost fold of the two-point axis weight.
For every mutant the script runs tests/test_host_point_math.py, which compiles the
header for the host and compares it with the oracle, and reports whether it fails
("killed") or passes ("SURVIVED").

    python tests/mutants/run_kernel_mutants.py SCRATCH_DIR [name filter ...]

SCRATCH_DIR receives a copy of oracle/, tests/ and the package (Python files and CUDA
headers). The repository itself is never modified.
"""
import os
import shutil
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

MUT = [
    ("Ricci: -1/2 Lfull", "M.Ric[s] = fma(-0.5, Lfull[s], t);", "M.Ric[s] = fma(-0.25, Lfull[s], t);", 1),
    ("Ricci: pair sum", "Rp[i][p] = offd(p) ? R[i][spi(p)][spj(p)] + R[i][spj(p)][spi(p)]",
     "Rp[i][p] = offd(p) ? R[i][spi(p)][spj(p)]", 1),
    ("Ricci: 2 A_ii", "t = fma(sc2<1>(Rp[i][p]), Dl[i][p], t);", "t = fma(Rp[i][p], Dl[i][p], t);", 1),
    ("DDphir: sign of the connection term", "M.DDphir[s] = hzero(AX, s) ? -dd : fma(mhiW, HW[s], -dd);",
     "M.DDphir[s] = hzero(AX, s) ? -dd : fma(mhiW, HW[s], dd);", 1),
    ("Abar: sign of 2 alpha DDphir", "double t = fma(-al2, DDphir[s], -DDal[s]);",
     "double t = fma(al2, DDphir[s], -DDal[s]);", 1),
    ("Lambda: 2 d alpha", "wl[k] = k == AX ? 0.0 : fma(al12, dphi[k], -sc2<1>(dal[k]));",
     "wl[k] = k == AX ? 0.0 : fma(al12, dphi[k], -dal[k]);", 1),
    ("advko: two-point centre fold", "W.c0 = AX >= 0 ? c0 - W.cax : c0;", "W.c0 = c0;", 2),
    ("dvz: wrong component", "return FAM == FAM_CYL && AX == 1 && k == 1 && i == 2;",
     "return FAM == FAM_CYL && AX == 1 && k == 1 && i == 1;", 1),
    ("dlz: wrong pair", "return FAM == FAM_CYL && AX == 1 && k == 2 && s == 4;",
     "return FAM == FAM_CYL && AX == 1 && k == 2 && s == 3;", 1),
    ("ddbz: wrong pair", "(kl == 1 || kl == 4)", "(kl == 1 || kl == 3)", 1),
    ("Delta_kij: surviving term", "Dl[k][s] = sc2<-1>(Dh[i][sp(k, k)]);", "Dl[k][s] = sc2<-1>(Dh[j][sp(k, k)]);", 1),
    ("gdiv: two-point skip", "if (AX < 0 || (l == AX) == (m == AX)) {", "if (AX < 0 || l != AX) {", 1),
]


def main():
    if len(sys.argv) < 2:
        sys.exit(__doc__)
    work = os.path.abspath(sys.argv[1])
    if work == ROOT:
        sys.exit("SCRATCH_DIR must not be the repository itself")
    only = sys.argv[2:]
    for d in ("oracle", "tests", "paper_2505_00097_gb300"):
        shutil.rmtree(os.path.join(work, d), ignore_errors=True)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(work, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(work, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    pkg = os.path.join(work, "paper_2505_00097_gb300")
    os.makedirs(os.path.join(pkg, "csrc"))
    for f in os.listdir(os.path.join(ROOT, "paper_2505_00097_gb300")):
        if f.endswith(".py"):
            shutil.copy(os.path.join(ROOT, "paper_2505_00097_gb300", f), pkg)
    for f in os.listdir(os.path.join(ROOT, "paper_2505_00097_gb300", "csrc")):
        if f.endswith((".cuh", ".h")):
            shutil.copy(os.path.join(ROOT, "paper_2505_00097_gb300", "csrc", f), os.path.join(pkg, "csrc"))
    src = os.path.join(pkg, "csrc", "bssn_point.cuh")
    orig = open(src).read()
    survivors = []
    for name, old, new, count in MUT:
        if only and not any(o in name for o in only):
            continue
        assert orig.count(old) == count, (name, orig.count(old))
        open(src, "w").write(orig.replace(old, new))
        t0 = time.time()
        r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_host_point_math.py", "-x", "-q",
                            "-p", "no:cacheprovider"], cwd=work, capture_output=True, text=True)
        first = next((ln.split("::")[-1][:70] for ln in r.stdout.splitlines() if ln.startswith("FAILED")), "")
        killed = r.returncode != 0
        print(f"{'killed  ' if killed else 'SURVIVED'} {time.time() - t0:5.1f}s  {name:36s} {first}", flush=True)
        if not killed:
            survivors.append(name)
    open(src, "w").write(orig)
    print("survivors:", survivors)
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main())
