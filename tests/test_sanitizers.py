"""Host sanitizers (compute-sanitizer is closed on this machine; these cover the
host code): the oracle compiled with AddressSanitizer and
UndefinedBehaviorSanitizer (gcc -fsanitize=address,undefined, every report
fatal) and run through a small C driver over the edge cases of its inputs --
n = 1 and 2, m = 0, d = 0, d >= n - 1, mixed arities, one sample, a
non-uniform order prior and family weights, a modular feature, and the two
zeta transforms on their own.  Any out-of-bounds access, leak, signed
overflow or other undefined behaviour fails the test."""
import os
import shutil
import sys
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int64_t orc_num_families(int n, int d);
int64_t orc_family_list(int n, int d, int i, uint32_t* masks);
int orc_upzeta(int n, int d, const double* s, double* t);
int orc_downzeta(int n, int d, const double* s, double* t);
int orc_edge_posteriors_ext(int n, int d, int m, const uint8_t* data, const uint8_t* arity,
                            double ess, const double* log_rho, const double* log_q,
                            const double* log_w, double* post, double* log_PD, double* A_out,
                            double* F_out, double* R_out, double* Gamma_out, double* logB_out,
                            uint32_t* mask_out);
int orc_feature_posterior(int n, int d, int m, const uint8_t* data, const uint8_t* arity,
                          double ess, const double* log_rho, const double* log_q,
                          const double* log_w, const double* log_f, double* p, double* log_PfD);

static uint64_t st = 88172645463325252ull;
static uint32_t rnd(void) { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (uint32_t)st; }

static int one(int n, int d, int m, int maxar, int priors)
{
    uint8_t ar[32];
    for (int i = 0; i < n; i++) ar[i] = (uint8_t)(1 + rnd() % maxar);
    uint8_t* data = (uint8_t*)malloc((size_t)m * n + 1);
    for (int s = 0; s < m; s++)
        for (int i = 0; i < n; i++) data[(size_t)s * n + i] = (uint8_t)(rnd() % ar[i]);
    int dd = d > n - 1 ? n - 1 : d;
    int64_t K = orc_num_families(n, d);
    double* post = (double*)calloc((size_t)n * n, sizeof(double));
    double lpd = 0.0;
    size_t N = (size_t)1 << n;
    double* A = (double*)malloc((size_t)n * N * sizeof(double));
    double* F = (double*)malloc(N * sizeof(double));
    double* R = (double*)malloc(N * sizeof(double));
    double* G = (double*)malloc((size_t)n * K * sizeof(double));
    double* lb = (double*)malloc((size_t)n * K * sizeof(double));
    uint32_t* mk = (uint32_t*)malloc((size_t)n * K * sizeof(uint32_t));
    double* lq = NULL; double* lw = NULL; double lr[40];
    for (int k = 0; k <= dd; k++) lr[k] = -0.3 * k;
    if (priors) {
        lq = (double*)malloc((size_t)n * n * sizeof(double));
        lw = (double*)malloc((size_t)n * K * sizeof(double));
        for (int x = 0; x < n * n; x++) lq[x] = -0.01 * (x % 7);
        for (int64_t x = 0; x < n * K; x++) lw[x] = (x % 5 == 0) ? -INFINITY : 0.1 * (x % 3);
        for (int i = 0; i < n; i++) lw[(size_t)i * K] = 0.0;     /* the empty parent set */
    }
    int rc = orc_edge_posteriors_ext(n, d, m, data, ar, 1.0, lr, lq, lw, post, &lpd, A, F, R, G,
                                     lb, mk);
    if (rc) { fprintf(stderr, "rc %d for n=%d d=%d m=%d\n", rc, n, d, m); return 1; }
    for (int x = 0; x < n * n; x++)
        if (!(post[x] >= -1e-12 && post[x] <= 1 + 1e-12)) { fprintf(stderr, "bad p\n"); return 1; }
    double* lf = (double*)malloc((size_t)n * K * sizeof(double));
    for (int64_t x = 0; x < n * K; x++) lf[x] = (x % 4 == 1) ? -INFINITY : 0.0;
    double p = 0.0, l2 = 0.0;
    rc = orc_feature_posterior(n, d, m, data, ar, 1.0, lr, lq, lw, lf, &p, &l2);
    if (rc || !(p >= -1e-12 && p <= 1 + 1e-12)) { fprintf(stderr, "feature\n"); return 1; }
    uint32_t* fl = (uint32_t*)malloc((size_t)K * sizeof(uint32_t));
    if (orc_family_list(n, d, n - 1, fl) != K) { fprintf(stderr, "families\n"); return 1; }
    double* s = (double*)malloc(N * sizeof(double));
    double* t = (double*)malloc(N * sizeof(double));
    for (size_t x = 0; x < N; x++) s[x] = -(double)(rnd() % 100) / 7.0;
    if (orc_upzeta(n, dd, s, t) || orc_downzeta(n, dd, s, t)) { fprintf(stderr, "zeta\n"); return 1; }
    free(data); free(post); free(A); free(F); free(R); free(G); free(lb); free(mk);
    free(lq); free(lw); free(lf); free(fl); free(s); free(t);
    return 0;
}

int main(void)
{
    static const int cases[][5] = {
        {1, 0, 5, 2, 0}, {1, 3, 0, 3, 0}, {2, 1, 1, 2, 0}, {3, 0, 10, 3, 1}, {4, 5, 0, 2, 1},
        {5, 2, 30, 4, 1}, {6, 3, 50, 3, 0}, {7, 6, 20, 2, 1}, {8, 2, 100, 5, 0}, {9, 3, 64, 2, 1},
    };
    for (size_t c = 0; c < sizeof cases / sizeof cases[0]; c++)
        if (one(cases[c][0], cases[c][1], cases[c][2], cases[c][3], cases[c][4])) return 1;
    puts("ok");
    return 0;
}
"""


def test_oracle_under_address_and_ub_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not found")
    drv = tmp_path / "driver.c"
    drv.write_text(DRIVER)
    exe = tmp_path / "oracle_asan"
    cmd = [gcc, "-std=c11", "-O1", "-g", "-fno-omit-frame-pointer",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           os.path.join(ROOT, "oracle", "bn_oracle.c"), str(drv), "-o", str(exe), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr and "cannot find" in r.stderr:
        pytest.skip("sanitizer runtime not installed")
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=600)
    assert run.returncode == 0, run.stderr[-4000:]
    assert "runtime error" not in run.stderr and "AddressSanitizer" not in run.stderr
    assert run.stdout.strip() == "ok"


def sanitizer_env():
    """LD_PRELOAD of gcc's ASan and UBSan runtimes (the Python process is not
    instrumented, the library is), or None when gcc has no such runtime."""
    gcc = shutil.which("gcc")
    if not gcc:
        return None
    libs = []
    for name in ("libasan.so", "libubsan.so"):
        p = subprocess.run([gcc, f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
        if not os.path.isabs(p) or not os.path.exists(p):
            return None
        libs.append(p)
    return dict(os.environ, LD_PRELOAD=":".join(libs), BN_ASAN="1", BN_TESTING="1",
                ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0:alloc_dealloc_mismatch=0",
                UBSAN_OPTIONS="print_stacktrace=1")


def run_under_sanitizers(tests, marker):
    from paper_1408_1664_gb300 import build as Bld
    env = sanitizer_env()
    if env is None:
        pytest.skip("no sanitizer runtime")
    Bld.build_asan()
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           "-m", marker] + tests
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    out = r.stdout + r.stderr
    print(out[-3000:])
    assert r.returncode == 0
    assert "AddressSanitizer" not in out and "runtime error:" not in out


def test_runtime_host_code_under_sanitizers():
    """The library's host code (validation, planning, layouts, the ABI's
    argument checks) built with ASan and UBSan, driven by the host tests."""
    run_under_sanitizers(["tests/test_host_planning.py", "tests/test_abi.py"], "not gpu")
