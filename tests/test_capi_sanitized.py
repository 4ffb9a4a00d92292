"""The library's host code under AddressSanitizer and UndefinedBehaviorSanitizer
(compute-sanitizer is not available for the device code).  Every CUDA source is
compiled for sm_103a with the host side instrumented and linked, with the CUDA
runtime, into a C driver.  The driver runs every entry point that needs no GPU:
  - the size queries over many sizes, both float types and every flag and knob;
  - pc_stream_info on a well-formed header, on every truncation of it, on
    single-byte corruptions of it and on 20,000 random headers, each passed in a
    heap block of exactly its length, so that an over-read is caught;
  - the launch-knob class table: tuned-config queries, and imports and exports
    of valid, invalid and table-filling entries;
  - argument errors of the compute entry points, which must return before any
    device work;
  - status strings and kernel-trace queries.
Any sanitizer report fails the test."""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2404_02826_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

DRIVER = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "pc.h"

static int failures = 0;
#define EXPECT(cond) do { if (!(cond)) { printf("FAIL line %d: %s\n", __LINE__, #cond); ++failures; } } while (0)

static uint64_t st = 0x9E3779B97F4A7C15ull;
static uint64_t rnd(void) { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return st; }

static void put_u16(unsigned char *h, int at, uint16_t v) { memcpy(h + at, &v, 2); }
static void put_u32(unsigned char *h, int at, uint32_t v) { memcpy(h + at, &v, 4); }
static void put_u64(unsigned char *h, int at, uint64_t v) { memcpy(h + at, &v, 8); }
static void put_f64(unsigned char *h, int at, double v) { memcpy(h + at, &v, 8); }

/* a header as the stream format describes it: 1000 float32 particles, 4 leaves */
static void good_header(unsigned char *h) {
    memset(h, 0, PC_HEADER_BYTES);
    memcpy(h, "PCB1", 4);
    put_u16(h, 4, 1);
    h[6] = PC_F32;
    h[7] = PC_EB_REL;
    put_u64(h, 8, 1000);
    put_f64(h, 16, 1e-3);
    put_f64(h, 24, 0.256);
    put_f64(h, 32, 0.5);
    put_f64(h, 40, 0.0);
    put_f64(h, 48, 1.0);
    put_f64(h, 56, 2.0);
    put_u64(h, 64, 4);
    put_u64(h, 72, 100);
    put_u32(h, 80, 250);
}

/* pc_stream_info on a heap copy of exactly len bytes */
static int info_of(const unsigned char *src, uint64_t len, pc_info *info) {
    unsigned char *p = (unsigned char *)malloc(len ? len : 1);
    if (len) memcpy(p, src, len);
    int rc = pc_stream_info(len ? p : NULL, len, info);
    free(p);
    return rc;
}

int main(void) {
    /* size queries */
    const uint64_t ns[] = {0, 1, 2, 3, 17, 1000, 4097, 65536, 1000003, 1u << 27, PC_MAX_PARTICLES};
    const uint32_t leaves[] = {0, 1, 16, 100, 4096, PC_MAX_LEAF_SIZE};
    const uint32_t flag_sets[] = {0, PC_FLAG_AUTOTUNE_LEAF, PC_FLAG_BOX_REDUCTION, PC_FLAG_REORDER,
                                  PC_FLAG_WIDEST_AXIS, PC_FLAG_AUTOTUNE_KNOBS, 31u};
    for (unsigned a = 0; a < sizeof ns / sizeof ns[0]; ++a)
        for (int dt = 0; dt < 2; ++dt)
            for (unsigned b = 0; b < sizeof leaves / sizeof leaves[0]; ++b)
                for (unsigned c = 0; c < sizeof flag_sets / sizeof flag_sets[0]; ++c) {
                    pc_config cfg;
                    memset(&cfg, 0, sizeof cfg);
                    cfg.leaf_size = leaves[b];
                    cfg.flags = flag_sets[c];
                    cfg.warp_node_max = (uint32_t)(rnd() % (PC_MAX_WARP_NODE_MAX + 1));
                    cfg.warp_leaf_max = (uint32_t)(rnd() % (PC_MAX_LEAF_SIZE + 1));
                    uint64_t x = 0, y = 0, z = 0;
                    int r1 = pc_compress_bound(ns[a], dt, &cfg, &x);
                    int r2 = pc_compress_workspace_size(ns[a], dt, &cfg, (int)(rnd() & 1), &y);
                    int r3 = pc_compress_host_workspace_size(ns[a], dt, &cfg, &z);
                    EXPECT(r1 == r2 && r2 == r3);
                    EXPECT(r1 == PC_OK || r1 == PC_ERR_ARG);
                    if (r1 == PC_OK) EXPECT(x >= PC_HEADER_BYTES && y > 0 && z >= y);
                    pc_config out;
                    int tuned = -1;
                    int r4 = pc_tuned_config(ns[a], dt, &cfg, &out, &tuned);
                    if (cfg.flags & PC_FLAG_AUTOTUNE_KNOBS) EXPECT(r4 == r1);
                    else EXPECT(r4 == PC_ERR_ARG);
                }
    uint64_t x = 0;
    EXPECT(pc_compress_bound(PC_MAX_PARTICLES + 1, PC_F32, NULL, &x) == PC_ERR_ARG);
    EXPECT(pc_compress_bound(10, 7, NULL, &x) == PC_ERR_ARG);
    EXPECT(pc_compress_bound(10, PC_F32, NULL, NULL) == PC_ERR_ARG);
    EXPECT(pc_decompress_workspace_size(123456, &x) == PC_OK && x > 0);
    EXPECT(pc_decompress_host_workspace_size(123456, PC_F64, 4096, &x) == PC_OK);
    EXPECT(pc_decompress_host_workspace_size(123456, 9, 4096, &x) == PC_ERR_ARG);
    EXPECT(pc_leaf_size_sweep_workspace_size(1u << 20, PC_F32, 64, 12000, &x) == PC_OK);
    EXPECT(pc_leaf_size_sweep_workspace_size(1u << 20, PC_F32, 8, 12000, &x) == PC_ERR_ARG);

    /* batch sizing */
    pc_compress_item items[40];
    memset(items, 0, sizeof items);
    for (int i = 0; i < 40; ++i) {
        items[i].n = rnd() % 3000000;
        items[i].dtype = (int32_t)(rnd() & 1);
        items[i].eb_mode = PC_EB_REL;
        items[i].eb = 1e-3;
        items[i].leaf_size = (uint32_t)(i % 3 ? 0 : 256);
        items[i].flags = (uint32_t)(i % 4 == 0 ? PC_FLAG_AUTOTUNE_LEAF | PC_FLAG_AUTOTUNE_KNOBS : 0);
    }
    for (uint32_t lanes = 0; lanes < 20; lanes += 3) {
        EXPECT(pc_compress_batch_workspace_size(items, 40, lanes, &x) == PC_OK);
        EXPECT(pc_compress_batch_workspace_size(items, 0, lanes, &x) == PC_OK);
    }
    items[7].dtype = 5;
    EXPECT(pc_compress_batch_workspace_size(items, 40, 4, &x) != PC_OK);
    EXPECT(pc_compress_batch_workspace_size(NULL, 3, 4, &x) == PC_ERR_ARG);
    pc_decompress_item ditems[8];
    memset(ditems, 0, sizeof ditems);
    for (int i = 0; i < 8; ++i) ditems[i].n = rnd() % 5000000;
    EXPECT(pc_decompress_batch_workspace_size(ditems, 8, 0, &x) == PC_OK);
    EXPECT(pc_decompress_batch_workspace_size(NULL, 8, 0, &x) == PC_ERR_ARG);

    /* headers */
    unsigned char h[PC_HEADER_BYTES];
    pc_info info;
    good_header(h);
    EXPECT(info_of(h, PC_HEADER_BYTES, &info) == PC_OK);
    EXPECT(info.n == 1000 && info.num_leaves == 4 && info.payload_words == 100 && info.leaf_size == 250);
    EXPECT(info.total_bytes == 96 + 32 * 4 + 4 * 100);
    for (uint64_t len = 0; len < PC_HEADER_BYTES; ++len) EXPECT(info_of(h, len, &info) != PC_OK);
    for (int at = 0; at < PC_HEADER_BYTES; ++at)
        for (int bit = 0; bit < 8; ++bit) {
            unsigned char g[PC_HEADER_BYTES];
            memcpy(g, h, sizeof g);
            g[at] ^= (unsigned char)(1u << bit);
            int rc = info_of(g, sizeof g, &info);
            EXPECT(rc == PC_OK || rc == PC_ERR_CORRUPT);
        }
    int accepted = 0;
    for (int k = 0; k < 20000; ++k) {
        unsigned char g[PC_HEADER_BYTES + 16];
        good_header(g);
        for (int i = PC_HEADER_BYTES; i < PC_HEADER_BYTES + 16; ++i) g[i] = (unsigned char)rnd();
        int flips = 1 + (int)(rnd() % 12);
        for (int f = 0; f < flips; ++f) g[rnd() % PC_HEADER_BYTES] = (unsigned char)rnd();
        if (k % 4 == 0)
            for (int i = 0; i < PC_HEADER_BYTES; ++i) g[i] = (unsigned char)rnd();
        int rc = info_of(g, PC_HEADER_BYTES + (rnd() % 2) * 16, &info);
        EXPECT(rc == PC_OK || rc == PC_ERR_CORRUPT);
        accepted += rc == PC_OK;
    }
    EXPECT(pc_stream_info(NULL, 96, &info) == PC_ERR_ARG);
    EXPECT(pc_stream_info(h, 96, NULL) == PC_ERR_ARG);

    /* the launch-knob class table */
    EXPECT(pc_autotune_reset() == PC_OK);
    uint32_t count = 99;
    EXPECT(pc_autotune_export(NULL, 0, &count) == PC_OK && count == 0);
    EXPECT(pc_autotune_export(NULL, 4, &count) == PC_ERR_ARG);
    pc_tuned_class cls[300];
    memset(cls, 0, sizeof cls);
    int m = 0;
    for (uint32_t bits = 0; bits < 32; ++bits)
        for (int dt = 0; dt < 2; ++dt)
            for (uint32_t leaf = 0; leaf < 4; ++leaf) {
                cls[m].n_bits = bits;
                cls[m].dtype = dt;
                cls[m].leaf_size = leaf;
                cls[m].warp_node_max = 1 + (uint32_t)(rnd() % PC_MAX_WARP_NODE_MAX);
                cls[m].warp_leaf_max = 1 + (uint32_t)(rnd() % PC_MAX_LEAF_SIZE);
                ++m;
            }
    EXPECT(m == 256);
    EXPECT(pc_autotune_import(cls, 256) == PC_OK);
    pc_tuned_class back[256];
    EXPECT(pc_autotune_export(back, 256, &count) == PC_OK && count == 256);
    EXPECT(pc_autotune_export(back, 10, &count) == PC_OK && count == 256);
    cls[256] = cls[0];
    cls[256].leaf_size = 9;
    EXPECT(pc_autotune_import(cls, 257) == PC_ERR_CAPACITY);
    cls[256].reserved = 1;
    EXPECT(pc_autotune_import(cls + 256, 1) == PC_ERR_ARG);
    EXPECT(pc_autotune_import(NULL, 1) == PC_ERR_ARG);
    EXPECT(pc_autotune_import(NULL, 0) == PC_OK);
    for (int k = 0; k < 2000; ++k) {
        pc_tuned_class t;
        memset(&t, 0, sizeof t);
        t.n_bits = (uint32_t)(rnd() % 40);
        t.dtype = (int32_t)(rnd() % 3);
        t.device = (int32_t)(rnd() % 300) - 20;
        t.flags = (uint32_t)(rnd() % 40);
        t.leaf_size = (uint32_t)(rnd() % 13000);
        t.warp_node_max = (uint32_t)(rnd() % 70000);
        t.warp_leaf_max = (uint32_t)(rnd() % 13000);
        int rc = pc_autotune_import(&t, 1);
        EXPECT(rc == PC_OK || rc == PC_ERR_ARG || rc == PC_ERR_CAPACITY);
    }
    pc_config q;
    memset(&q, 0, sizeof q);
    q.flags = PC_FLAG_AUTOTUNE_KNOBS;
    pc_config got;
    int tuned = 0;
    EXPECT(pc_tuned_config(1000, PC_F32, &q, &got, &tuned) == PC_OK);
    EXPECT(pc_tuned_config(1000, PC_F32, &q, NULL, &tuned) == PC_ERR_ARG);
    EXPECT(pc_autotune_reset() == PC_OK);

    /* argument errors before any device work */
    EXPECT(pc_compress(NULL, 10, PC_F32, PC_EB_REL, 1e-3, NULL, NULL, 0, NULL, NULL, 0, NULL, NULL) == PC_ERR_ARG);
    EXPECT(pc_compress_noalloc(NULL, 10, PC_F32, PC_EB_REL, 1e-3, NULL, NULL, 0, NULL, NULL) == PC_ERR_ARG);
    EXPECT(pc_decompress_host(NULL, 0, NULL, 0, NULL, 0, NULL) == PC_ERR_ARG);
    EXPECT(pc_compress_host(NULL, 10, PC_F32, PC_EB_REL, 1e-3, NULL, NULL, 0, NULL, NULL, 0, NULL) == PC_ERR_ARG);
    EXPECT(pc_compress_batch(NULL, 3, 1, NULL, 0, NULL) != PC_OK);
    EXPECT(pc_decompress_batch(NULL, 3, 1, NULL, 0, NULL) == PC_ERR_ARG);
    EXPECT(pc_server_create(NULL, 0, 1, NULL) == PC_ERR_ARG);
    EXPECT(pc_leaf_size_sweep(NULL, 10, PC_F32, PC_EB_REL, 1e-3, 64, 128, NULL, 0, NULL, NULL, 0, NULL) != PC_OK);

    /* status strings, version, trace queries */
    for (int s = -3; s < 12; ++s) EXPECT(pc_error_string(s) != NULL && strlen(pc_error_string(s)) > 0);
    EXPECT(pc_format_version() == 1);
    EXPECT(pc_trace_reset() == PC_OK);
    EXPECT(pc_trace_count() == 0);
    const char *name = NULL;
    uint64_t launches = 0;
    double ms = 0;
    EXPECT(pc_trace_get(0, &name, &launches, &ms) != PC_OK);
    EXPECT(pc_trace_get(-1, &name, &launches, &ms) != PC_OK);

    printf("checked, %d random headers accepted, %d failures\n", accepted, failures);
    return failures ? 1 : 0;
}
"""


def _tool(name):
    for cand in (shutil.which(name), os.path.join("/usr/local/cuda/bin", name)):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_library_host_code_clean_under_sanitizers(tmp_path):
    nvcc, gcc, gxx = _tool("nvcc"), shutil.which("gcc"), shutil.which("g++")
    if not (nvcc and gcc and gxx):
        pytest.skip("nvcc, gcc and g++ are needed")
    cudalib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")
    san = "-fsanitize=address,-fsanitize=undefined,-fno-omit-frame-pointer,-fno-sanitize-recover=all"
    srcs = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))

    def one(src):
        obj = str(tmp_path / (src + ".o"))
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17", "-Xcompiler", san,
               "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(one, srcs))
    (tmp_path / "driver.c").write_text(DRIVER)
    drv = str(tmp_path / "driver.o")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                        "-I", INCLUDE, "-c", str(tmp_path / "driver.c"), "-o", drv], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    exe = str(tmp_path / "driver")
    r = subprocess.run([gxx, "-fsanitize=address,undefined", drv] + objs +
                       ["-L", cudalib, "-lcudart_static", "-ldl", "-lrt", "-lpthread", "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "0 failures" in out and "ERROR: AddressSanitizer" not in out and "runtime error" not in out, out[-4000:]
