"""The C-ABI library builds, loads and exports every entry point that
include/tauleap.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tauleap.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssa_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1309_7695_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ssa_load_model", "ssa_submit_batch", "ssa_poll", "ssa_fetch",
                     "ssa_simulate_dev", "ssa_release_job", "ssa_free_model", "ssa_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_binding_names_match_header(libpath):
    from paper_1309_7695_b300 import abi
    assert sorted(abi.EXPORTED) == declared_functions()


def test_host_side_validation_without_gpu(libpath):
    # model validation runs on the host before any CUDA call
    from paper_1309_7695_b300 import abi, inputs
    lib = abi.lib()
    assert lib.ssa_abi_version() == 1
    o = abi.ssa_default_options()
    assert o.eps == 0.03 and o.n_c == 10 and o.ssa_block == 100 and o.max_attempts == 10**8
    bad = inputs.Network(2, [[(0, 2), (1, 1)]], [[]])     # order 3
    with pytest.raises(abi.SsaError) as e:
        abi.Model(bad)
    assert e.value.code == abi.SSA_EINVAL and "order" in str(e.value)
    bad = inputs.Network(2, [[(5, 1)]], [[]])              # species out of range
    with pytest.raises(abi.SsaError) as e:
        abi.Model(bad)
    assert e.value.code == abi.SSA_EINVAL
