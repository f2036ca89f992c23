"""The oracle's pins catch plausible mistakes.

Each mutant below is a copy of oracle/tauleap_oracle.c with one planted
mistake of the kind a careful reader could still make (a wrong constant, a
wrong index, a dropped term, an off-by-one, a sign).  The copy is built with
the oracle's own flags and the pin tests (tests/test_oracle_*.py, minus the
10^8-input libm comparison, which repeats the ulp pins at scale) run against
it through the binding's ORACLE_LIBRARY override.  Every mutant must make
some pin fail.  The mistakes are planted on the CPU only; nothing here
touches the engine.

Left out on purpose: changes that alter no result of the method, so that no
test of the oracle's output could see them: a comparison turned from < into
<= where equality has probability zero (a uniform exactly on a cdf value, a
sample time equal to an event time), PTRS squeeze and hat constants (the
acceptance step keeps the law exact; they change which uniforms are used,
which the engine's bit-for-bit parity tests see), and the step-size
constants of the ODE controller (the solution stays within tolerance)."""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tauleap_oracle.c")
PIN_FILES = ["test_oracle_primitives.py", "test_oracle_poisson.py", "test_oracle_simulation.py",
             "test_oracle_cle.py", "test_oracle_rre.py"]

# (name, text in the oracle, replacement)
MUTANTS = [
    # Philox4x32-10 and the uniform
    ("philox round multiplier", "(uint64_t)0xD2511F53u * (uint64_t)c0", "(uint64_t)0xD2511F55u * (uint64_t)c0"),
    ("philox key increment", "k0 += 0x9E3779B9u;", "k0 += 0x9E3779BBu;"),
    ("u01 offset", "return ((double)m + 0.5) * 0x1p-52;", "return ((double)m + 0.25) * 0x1p-52;"),
    ("philox round count", "for (int round = 0; round < 10; ++round) {", "for (int round = 0; round < 9; ++round) {"),
    ("philox output words swapped", "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi0 ^ c1 ^ k0;"),
    ("u01 keeps 53 bits", "| (uint64_t)w1) >> 12;", "| (uint64_t)w1) >> 11;"),
    # ln, exp, ln k!
    ("ln polynomial coefficient", "    p = p * r + 1.0 / 3.0;\n    p = p * r - 1.0 / 2.0;",
     "    p = p * r + 1.0 / 4.0;\n    p = p * r - 1.0 / 2.0;"),
    ("ln low part sign", "double lo = ((de * LN2_LO + LOG_LO[j]) + err) + q;",
     "double lo = ((LOG_LO[j] - de * LN2_LO) + err) + q;"),
    ("exp Taylor coefficient", "p = p * r + 1.0 / 24.0;", "p = p * r + 1.0 / 25.0;"),
    ("exp reduction sign", "double r = (x - n * LN2_HI) - n * LN2_LO;", "double r = (x - n * LN2_HI) + n * LN2_LO;"),
    ("ln k! Stirling term sign", "ser = ser * r2 - 1.0 / 360.0;", "ser = ser * r2 + 1.0 / 360.0;"),
    ("ln k! Stirling from k = 2", "    if (k < 10) {\n        double f = 1.0;", "    if (k < 2) {\n        double f = 1.0;"),
    ("ln k! exact product bound", "for (int64_t i = 2; i <= k; ++i) f = f * (double)i;",
     "for (int64_t i = 2; i < k; ++i) f = f * (double)i;"),
    # Poisson sampler
    ("inversion recurrence index", "p = (p * lam) * (1.0 / (double)k);", "p = (p * lam) * (1.0 / (double)(k + 1));"),
    ("PTRS log-pmf off by one", "double rhs = -lam + kd * loglam - oracle_lnfact((int64_t)kd);",
     "double rhs = -lam + kd * loglam - oracle_lnfact((int64_t)kd + 1);"),
    ("PTRS log-pmf uses sqrt", "double rhs = -lam + kd * loglam - oracle_lnfact((int64_t)kd);",
     "double rhs = -lam + kd * slam - oracle_lnfact((int64_t)kd);"),
    ("PTRS rejects k = 0", "if (kd < 0.0 || (us < 0.013 && V > us)) continue;",
     "if (kd <= 0.0 || (us < 0.013 && V > us)) continue;"),
    # Langevin increment
    ("Langevin threshold", "#define CLE_MIN_MEAN 1000.0", "#define CLE_MIN_MEAN 100.0"),
    ("polar method drops /s", "double z = v1 * sqrt((-2.0 * oracle_log(s)) / s);",
     "double z = v1 * sqrt(-2.0 * oracle_log(s));"),
    ("Langevin increment scale", "double k = floor((lam + sqrt(lam) * z) + 0.5);", "double k = floor((lam + lam * z) + 0.5);"),
    # propensities
    ("2X propensity without the -1", "return c * (double)((xi * (xi - 1)) / 2);", "return c * (double)((xi * xi) / 2);"),
    ("X+Y propensity index", "case 2: return (c * (double)x[m->r_sp0[j]]) * (double)x[m->r_sp1[j]];",
     "case 2: return (c * (double)x[m->r_sp0[j]]) * (double)x[m->r_sp0[j]];"),
    # critical set and tau'
    ("critical threshold off by one", "L < (int64_t)o->n_c);", "L <= (int64_t)o->n_c);"),
    ("critical test ignores a_j > 0", "w->crit[j] = (w->a[j] > 0.0 && L < (int64_t)o->n_c);",
     "w->crit[j] = (L < (int64_t)o->n_c);"),
    ("mu uses nu squared", "w->mu[i] = w->mu[i] + (double)nv * w->a[j];", "w->mu[i] = w->mu[i] + (double)(nv * nv) * w->a[j];"),
    ("sigma^2 term without the square of the bound", "double t2 = (bound * bound) / w->sig2[i];",
     "double t2 = bound / w->sig2[i];"),
    ("bound multiplies by g", "double bound = (o->eps * xd) / g;", "double bound = (o->eps * xd) * g;"),
    ("g of an X+Y reactant", "case 2: g = 2.0; break;", "case 2: g = 1.0; break;"),
    ("g of a 2X reactant", "g = (x[i] >= 2) ? 2.0 + 1.0 / (xd - 1.0) : 2.0;", "g = (x[i] >= 2) ? 2.0 + 1.0 / xd : 2.0;"),
    ("second reactant left out of I_rs", "if (kind == 2) w->irs[m->r_sp1[j]] = 1;", ";"),
    # leap
    ("tau'' divides by a0", "double tau2 = (a0c > 0.0) ? -oracle_log(u_tau) / a0c : INFINITY;",
     "double tau2 = (a0c > 0.0) ? -oracle_log(u_tau) / a0 : INFINITY;"),
    ("critical firing ignores the sample time", "if (tau2 <= tau1 && tau2 <= delta) {", "if (tau2 <= tau1) {"),
    ("critical reaction never fires in a leap", "w->k[j] = (j == jc) ? 1 : 0; continue;", "w->k[j] = 0; continue;"),
    ("leap update ignores k", "w->xnew[m->nu_sp[e]] += w->k[j] * (int64_t)m->nu_val[e];",
     "w->xnew[m->nu_sp[e]] += (int64_t)m->nu_val[e];"),
    ("a leap to zero counts as negative", "if (w->xnew[i] < 0) neg = 1;", "if (w->xnew[i] <= 0) neg = 1;"),
    ("SSA fallback threshold", "if (do_ssa || tau1 < o->ssa_factor / a0) {", "if (do_ssa || tau1 < o->ssa_factor * a0) {"),
    # exact SSA step
    ("SSA selection reuses the time uniform", "int jf = canon_select(w->a, M, levels, u2 * a0);",
     "int jf = canon_select(w->a, M, levels, u1 * a0);"),
    ("SSA waiting time uses a0 squared", "double tau = -oracle_log(u1) / a0;", "double tau = -oracle_log(u1) / (a0 * a0);"),
    # canonical sum and selection
    ("slot tree partner", "levels[k][l] = levels[k - 1][l] + levels[k - 1][l ^ d];",
     "levels[k][l] = levels[k - 1][l] + levels[k - 1][l ^ (d >> 1)];"),
    ("selection keeps the left mass", "            target = target - left;\n", "\n"),
    # reaction-rate equations
    ("Dormand-Prince weight", "DP_B3 = 500.0 / 1113.0", "DP_B3 = 500.0 / 1112.0"),
    ("Dormand-Prince FSAL derivative not carried", "{ x[i] = xn[i]; k[1][i] = k[7][i]; }", "{ x[i] = xn[i]; }"),
    ("mean-field 2X rate", "default: a[j] = c[j] * ((x[m->r_sp0[j]] * x[m->r_sp0[j]]) * 0.5); break;",
     "default: a[j] = c[j] * (x[m->r_sp0[j]] * x[m->r_sp0[j]]); break;"),
]


def _run_mutant(index, workdir):
    name, before, after = MUTANTS[index]
    from oracle import build as oracle_build

    src = open(SRC).read()
    mutated = src.replace(before, after, 1)
    c_path = os.path.join(workdir, f"mutant{index}.c")
    so_path = os.path.join(workdir, f"libmutant{index}.so")
    with open(c_path, "w") as f:
        f.write(mutated)
    oracle_build.compile_source(c_path, so_path)
    env = dict(os.environ, ORACLE_LIBRARY=so_path, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-k", "not 1e8"] + \
          [os.path.join(ROOT, "tests", f) for f in PIN_FILES]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, cwd=ROOT, timeout=900)
    failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
    return name, r.returncode, failed[:1]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(SRC).read()
    for name, before, _ in MUTANTS:
        assert src.count(before) == 1, f"mutation site of '{name}' not found exactly once"
    workers = max(1, min(6, (os.cpu_count() or 2) // 2))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda i: _run_mutant(i, str(tmp_path)), range(len(MUTANTS))))
    survivors = [name for name, rc, _ in results if rc == 0]
    errors = [(name, rc) for name, rc, _ in results if rc not in (0, 1)]
    assert not errors, f"pin runs that did not complete: {errors}"
    assert not survivors, f"planted mistakes no pin catches: {survivors}"
