"""Host-only checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function include/ah.h declares, and the ctypes
structs of the binding match the C layouts."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1809_00995_gb300 as ah

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ah.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ah_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    lib = ah.load()
    names = declared_functions()
    assert "ah_create" in names and "ah_step" in names and "ah_observables" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(ah.exported_symbols())
    out = subprocess.run(["nm", "-D", "--defined-only", ah.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ah_\w+)", out))
    assert set(names) <= exported


def test_abi_version_and_struct_layouts(tmp_path):
    assert ah.ah_abi_version() == 6
    src = tmp_path / "sz.c"
    src.write_text('#include "ah.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(ah_config), sizeof(ah_obs),'
                   ' sizeof(ah_info), offsetof(ah_obs, sums), offsetof(ah_obs, nonfinite),'
                   ' offsetof(ah_config, seed), offsetof(ah_info, variant_name), sizeof(ah_sums), sizeof(ah_batch_stats),'
                   ' sizeof(ah_server_stats), sizeof(ah_window), offsetof(ah_window, out),'
                   ' offsetof(ah_info, fused_diag_passes), offsetof(ah_info, weak_field_launches));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(ah.ah_config), ctypes.sizeof(ah.ah_obs), ctypes.sizeof(ah.ah_info),
            ah.ah_obs.sums.offset, ah.ah_obs.nonfinite.offset, ah.ah_config.seed.offset,
            ah.ah_info.variant_name.offset, ctypes.sizeof(ah.ah_sums), ctypes.sizeof(ah.ah_batch_stats),
            ctypes.sizeof(ah.ah_server_stats), ctypes.sizeof(ah.ah_window), ah.ah_window.out.offset,
            ah.ah_info.fused_diag_passes.offset, ah.ah_info.weak_field_launches.offset]
    assert got == want


def test_config_defaults_without_gpu():
    c = ah.ah_config_default(64)
    assert (c.N, c.era, c.precision, c.dx, c.dt, c.lambda0, c.e0, c.sigma) == (64, 1, 0, 0.5, 0.1, 2.0, 1.0, 1.0)
    assert c.tau_end == 16.0 and c.tau_ref == 16.0 and c.tau0 == 1.0


def test_binding_constants_match_the_header():
    """Every enum constant of include/ah.h has the same value in the binding."""
    import re
    hdr = open(HEADER).read()
    found = 0
    for body in re.findall(r"enum\s*(?:\w+\s*)?\{([^}]*)\}", hdr):
        for name, val in re.findall(r"(AH_\w+)\s*=\s*(\d+)", body):
            assert getattr(ah, name) == int(val), name
            found += 1
    assert found >= 20 and ah.AH_FLAG_WRAP_THETA == 4


def test_two_step_flag_refused_for_fp64_and_plain_without_gpu():
    """AH_FLAG_TWO_STEP is an FP32 fused-kernel mode: other configurations are
    refused by the argument check, before any device call."""
    for prec, kern in [(ah.AH_FP64, ah.AH_KERNEL_FUSED), (ah.AH_FP32, ah.AH_KERNEL_PLAIN)]:
        c = ah.config(8, precision=prec, kernel=kern, flags=ah.AH_FLAG_TWO_STEP)
        with pytest.raises(ah.AhError) as e:
            ah.ah_create_ex(c)
        assert e.value.status == ah.AH_ERR_ARG and "TWO_STEP" in str(e.value)
