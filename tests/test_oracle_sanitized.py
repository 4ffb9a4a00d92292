"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (host side;
compute-sanitizer is not available for the CUDA path).  A small C driver,
compiled together with oracle/oracle.c, runs every entry point the tests use:
compression and decoding (both float types, both bounds), the bit-box reduction
in both orders, the reordering, the widest-cell rule, and decoding of
malformed streams, which must be rejected without a memory error."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")

DRIVER = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int oracle_compress_rule(const void *, uint64_t, int, int, double, uint64_t, int, uint8_t **, uint64_t *, uint64_t **);
int oracle_compress_reduced(const void *, uint64_t, int, int, double, uint64_t, int, int, uint8_t **, uint64_t *,
                            uint64_t **, uint64_t *);
int oracle_reorder(const uint8_t *, uint64_t, const uint64_t *, uint8_t **, uint64_t *, uint64_t *, int *);
int oracle_decompress(const uint8_t *, uint64_t, void *, uint64_t);
void oracle_free(void *);

static uint64_t st = 88172645463325252ull;
static double rnd(void) { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (double)(st >> 11) / 9007199254740992.0; }

static int round_trip(const void *pos, uint64_t n, int dtype, int mode, double eb, uint64_t r, int variant)
{
    uint8_t *s = NULL, *s2 = NULL;
    uint64_t bytes = 0, bytes2 = 0, *perm = NULL, rounds = 0;
    int rc;
    if (variant == 0 || variant == 1)
        rc = oracle_compress_rule(pos, n, dtype, mode, eb, r, variant, &s, &bytes, &perm);
    else
        rc = oracle_compress_reduced(pos, n, dtype, mode, eb, r, 0, variant == 3, &s, &bytes, &perm, &rounds);
    if (rc) return 100 + rc;
    uint64_t *perm2 = malloc((n ? n : 1) * sizeof(uint64_t));
    int order[3];
    rc = oracle_reorder(s, bytes, perm, &s2, &bytes2, perm2, order);
    if (rc) return 200 + rc;
    size_t esz = dtype ? 8 : 4;
    void *dec = malloc((n ? n : 1) * 3 * esz);
    rc = oracle_decompress(s2, bytes2, dec, n * 3 * esz);
    if (rc) return 300 + rc;
    /* truncated and corrupted copies are rejected */
    for (uint64_t cut = 0; cut < bytes2; cut += bytes2 / 7 + 1)
        if (oracle_decompress(s2, cut, dec, n * 3 * esz) == 0 && cut < bytes2) return 400;
    uint8_t *bad = malloc(bytes2);
    memcpy(bad, s2, bytes2);
    if (bytes2 > 100) bad[96 + 28] = 40; /* a width above 31 */
    if (bytes2 > 100 && oracle_decompress(bad, bytes2, dec, n * 3 * esz) == 0) return 401;
    free(bad);
    free(dec);
    free(perm2);
    oracle_free(s);
    oracle_free(s2);
    oracle_free(perm);
    return 0;
}

int main(void)
{
    const uint64_t n = 6000;
    float *pf = malloc(n * 3 * sizeof(float));
    double *pd = malloc(n * 3 * sizeof(double));
    for (uint64_t i = 0; i < 3 * n; i++) {
        double c = (i / 3) % 5 * 40.0;
        pd[i] = c + rnd() * (i % 3 == 0 ? 8.0 : 2.0);
        pf[i] = (float)pd[i];
    }
    for (int variant = 0; variant < 4; variant++)
        for (int r = 1; r <= 700; r += 233) {
            int rc = round_trip(pf, n, 0, 1, 1e-3, (uint64_t)r, variant);
            if (!rc) rc = round_trip(pd, n, 1, 0, 1e-4, (uint64_t)r, variant);
            if (!rc) rc = round_trip(pf, 1, 0, 1, 1e-3, (uint64_t)r, variant);
            if (rc) { printf("failed %d (variant %d, r %d)\n", rc, variant, r); return 1; }
        }
    free(pf);
    free(pd);
    puts("ok");
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_oracle_clean_under_sanitizers(tmp_path):
    drv = tmp_path / "driver.c"
    drv.write_text(DRIVER)
    exe = tmp_path / "driver"
    cmd = ["gcc", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-Wno-unknown-pragmas", str(drv), ORACLE, "-o", str(exe), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtime unavailable: " + r.stderr.splitlines()[0])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.stdout[-2000:], r.stderr[-4000:])
    assert "runtime error" not in r.stderr and "ERROR: AddressSanitizer" not in r.stderr
