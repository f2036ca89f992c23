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
    assert lib.ssa_abi_version() == 2
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


def test_new_entry_points_reject_null_handles_without_gpu(libpath):
    # argument checks of the sweep-moments, RRE and multi-network entry points
    # run before any CUDA call, so they answer on a machine without a GPU
    import ctypes

    from paper_1309_7695_b300 import abi
    lib = abi.lib()
    o = abi.ssa_default_options()
    rc = lib.ssa_simulate_moments_dev(None, 4, 0, None, None, 1.0, None, 2, 0, ctypes.byref(o), None, None, None, None)
    assert rc == abi.SSA_EINVAL and b"model" in lib.ssa_last_error()
    rc = lib.ssa_integrate_rre_dev(None, 4, None, None, None, 2, 1e-8, 1e-8, 100, None, None, None)
    assert rc == abi.SSA_EINVAL
    rc = lib.ssa_simulate_multi_dev(-1, None, ctypes.byref(o), None)
    assert rc == abi.SSA_EINVAL
    o.mode = 7
    rc = lib.ssa_simulate_multi_dev(1, (abi.Group * 1)(), ctypes.byref(o), None)
    assert rc == abi.SSA_EINVAL and b"mode" in lib.ssa_last_error()
    assert abi.SSA_MODE_CLE == 2
