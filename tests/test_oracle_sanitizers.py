"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU): a
small C driver compiled together with oracle/ah_oracle.c runs every entry point
(initialisation of the lattice and of windows, stepping with each option,
whole-lattice and box diagnostics, energy, gauge transform, windings) on small
odd lattices; any out-of-bounds access, leak or undefined operation fails."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r'''
#include "%s"
#include <stdio.h>

static uint64_t lcg = 12345u;
static double rnd(void) { lcg = lcg * 6364136223846793005ull + 1442695040888963407ull; return (double)(lcg >> 11) * 0x1p-53 - 0.5; }

int main(void)
{
    const int64_t sizes[3] = { 4, 5, 7 };
    for (int k = 0; k < 3; ++k) {
        const int64_t M = sizes[k], M3 = M * M * M;
        for (int flags = 0; flags < 4; ++flags) {
            aho_params p = { 2 * M, 0.5, 0.1, 1 + (flags & 1), flags, -0.5, 2.0, 1.0, 1.0, 1.0, 1.35, 7u };
            double *f = malloc(sizeof(double) * 10 * M3);
            double *alpha = malloc(sizeof(double) * M3);
            int8_t *w = malloc(3 * M3);
            aho_init_box(&p, f, M, 1, 2, 3);                       /* a window of the 2M lattice */
            for (int64_t s = 2 * M3; s < 10 * M3; ++s) f[s] = 3.0 * rnd();
            if (aho_evolve(&p, f, M, 0, 6) != 0) return 2;
            aho_diag_out o;
            aho_diag(&p, f, M, 6, 0, 0, 0, M, M, M, &o);
            aho_diag(&p, f, M, 6, 1, 1, 1, M - 2, M - 2, M - 2, &o);
            volatile double e = aho_energy(&p, f, M, 6);
            (void)e;
            for (int64_t s = 0; s < M3; ++s) alpha[s] = 4.0 * rnd();
            aho_gauge_transform(f, M, alpha);
            aho_windings(f, M, w);
            free(f); free(alpha); free(w);
        }
    }
    puts("ok");
    return 0;
}
'''


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    src = tmp_path / "driver.c"
    src.write_text(DRIVER % os.path.join(ROOT, "oracle", "ah_oracle.c"))
    exe = tmp_path / "driver"
    r = subprocess.run([gcc, "-std=gnu11", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=all", str(src), "-o", str(exe), "-lm"], capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtimes not available: " + r.stderr.splitlines()[0])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stderr[-2000:]
    assert "runtime error" not in run.stderr and "ERROR: AddressSanitizer" not in run.stderr
