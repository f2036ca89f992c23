"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

The oracle's source is built once more with -fsanitize=address,undefined
(errors fatal) and the pin tests run against that build through the
binding's ORACLE_LIBRARY override, with the sanitizer runtimes preloaded
into the Python process.  Any out-of-bounds access, use after free, signed
overflow, bad shift or misaligned load on the pins' paths (the simulation
loop with its status paths, the samplers, the canonical sums, the ODE
integrator) aborts the run."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["test_oracle_primitives.py", "test_oracle_poisson.py", "test_oracle_simulation.py",
             "test_oracle_cle.py", "test_oracle_rre.py"]


def _runtime(name):
    path = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_pins_pass_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if asan is None or ubsan is None:
        pytest.skip("sanitizer runtimes not installed")
    from oracle import build as oracle_build

    lib = str(tmp_path / "liboracle_sanitized.so")
    oracle_build.compile_source(oracle_build.SRC, lib, extra=["-g", "-fno-omit-frame-pointer",
                                                              "-fsanitize=address,undefined",
                                                              "-fno-sanitize-recover=all"])
    env = dict(os.environ, ORACLE_LIBRARY=lib, LD_PRELOAD=f"{asan} {ubsan}", OMP_NUM_THREADS="4",
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-k", "not 1e8 and not 1e7"] + \
          [os.path.join(ROOT, "tests", f) for f in PIN_FILES]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, cwd=ROOT, timeout=1800)
    report = [ln for ln in (r.stdout + r.stderr).splitlines()
              if "runtime error" in ln or "ERROR: AddressSanitizer" in ln]
    assert r.returncode == 0 and not report, (r.returncode, report[:5], r.stdout[-2000:])
