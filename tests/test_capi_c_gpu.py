"""The boundary from C on the GPU: a C99 program linked against the library and
the CUDA runtime, with its own cudaMalloc'd buffers and no Python in the data
path, compresses, decompresses, batches and serves two inputs (float32
cosmology-shaped at rel 1e-3, float64 fluid-shaped at abs 1e-4).  The streams
it writes must equal the oracle's byte for byte and the decoded positions the
oracle's decode, which also shows that the header's structs (pc_compress_item,
pc_request, pc_completion, pc_info) are read as the library lays them out.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")
pytestmark = pytest.mark.gpu

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <cuda_runtime.h>
#include "pc.h"

#define CK(x) do { int rc_ = (int)(x); if (rc_) { fprintf(stderr, "%s:%d: %s -> %d\n", __FILE__, __LINE__, #x, rc_); return 1; } } while (0)

typedef struct { uint64_t n; int dtype; int mode; double eb; void *host; void *dev; uint64_t bytes; } input;

static int load(const char *path, input *in) {
    FILE *f = fopen(path, "rb");
    if (!f) return 1;
    uint64_t hdr[2];
    if (fread(hdr, 8, 2, f) != 2) return 1;
    double eb;
    if (fread(&eb, 8, 1, f) != 1) return 1;
    in->n = hdr[0];
    in->dtype = (int)(hdr[1] & 0xff);
    in->mode = (int)(hdr[1] >> 8);
    in->eb = eb;
    in->bytes = in->n * 3 * (in->dtype == PC_F32 ? 4 : 8);
    in->host = malloc(in->bytes);
    if (fread(in->host, 1, in->bytes, f) != in->bytes) return 1;
    fclose(f);
    if (cudaMalloc(&in->dev, in->bytes)) return 1;
    return (int)cudaMemcpy(in->dev, in->host, in->bytes, cudaMemcpyHostToDevice);
}

static int save_dev(const char *dir, const char *name, const void *dev, uint64_t bytes) {
    char path[4096];
    snprintf(path, sizeof path, "%s/%s", dir, name);
    void *h = malloc(bytes ? bytes : 1);
    if (bytes && cudaMemcpy(h, dev, bytes, cudaMemcpyDeviceToHost)) return 1;
    FILE *f = fopen(path, "wb");
    if (!f) return 1;
    if (bytes && fwrite(h, 1, bytes, f) != bytes) return 1;
    fclose(f);
    free(h);
    return 0;
}

int main(int argc, char **argv) {
    if (argc != 4) return 2;
    const char *dir = argv[3];
    input in[2];
    CK(load(argv[1], &in[0]));
    CK(load(argv[2], &in[1]));
    void *stream_dev[2];
    uint64_t stream_size[2];
    char name[64];
    for (int k = 0; k < 2; ++k) {
        pc_config cfg;
        memset(&cfg, 0, sizeof cfg);
        uint64_t bound = 0, ws_bytes = 0, dws_bytes = 0;
        CK(pc_compress_bound(in[k].n, in[k].dtype, &cfg, &bound));
        CK(pc_compress_workspace_size(in[k].n, in[k].dtype, &cfg, 0, &ws_bytes));
        void *out = NULL, *ws = NULL;
        CK(cudaMalloc(&out, bound));
        CK(cudaMalloc(&ws, ws_bytes));
        uint64_t size = 0;
        CK(pc_compress(in[k].dev, in[k].n, in[k].dtype, in[k].mode, in[k].eb, &cfg, out, bound, &size, ws, ws_bytes,
                       NULL, NULL));
        snprintf(name, sizeof name, "stream%d.bin", k);
        CK(save_dev(dir, name, out, size));
        unsigned char hdr[96];
        CK(cudaMemcpy(hdr, out, sizeof hdr, cudaMemcpyDeviceToHost));
        pc_info info;
        CK(pc_stream_info(hdr, sizeof hdr, &info));
        printf("info %d %llu %d %llu %llu %u\n", k, (unsigned long long)info.n, (int)info.dtype,
               (unsigned long long)info.num_leaves, (unsigned long long)info.total_bytes, info.lossless_axes);
        CK(pc_decompress_workspace_size(info.n, &dws_bytes));
        void *dws = NULL, *dec = NULL;
        CK(cudaMalloc(&dws, dws_bytes));
        CK(cudaMalloc(&dec, in[k].bytes));
        CK(pc_decompress(out, size, dec, in[k].bytes, dws, dws_bytes, NULL));
        snprintf(name, sizeof name, "dec%d.bin", k);
        CK(save_dev(dir, name, dec, in[k].bytes));
        stream_dev[k] = out;
        stream_size[k] = size;
        CK(cudaFree(ws));
        CK(cudaFree(dws));
        CK(cudaFree(dec));
    }
    /* both inputs in one batch call */
    pc_compress_item items[2];
    memset(items, 0, sizeof items);
    for (int k = 0; k < 2; ++k) {
        items[k].positions = in[k].dev;
        items[k].n = in[k].n;
        items[k].dtype = in[k].dtype;
        items[k].eb_mode = in[k].mode;
        items[k].eb = in[k].eb;
        pc_config cfg;
        memset(&cfg, 0, sizeof cfg);
        CK(pc_compress_bound(in[k].n, in[k].dtype, &cfg, &items[k].out_capacity));
        CK(cudaMalloc(&items[k].out, items[k].out_capacity));
        items[k].status = -1;
    }
    uint64_t bws = 0;
    CK(pc_compress_batch_workspace_size(items, 2, 2, &bws));
    void *bw = NULL;
    CK(cudaMalloc(&bw, bws));
    CK(pc_compress_batch(items, 2, 2, bw, bws, NULL));
    for (int k = 0; k < 2; ++k) {
        printf("batch %d %d %llu\n", k, items[k].status, (unsigned long long)items[k].out_size);
        snprintf(name, sizeof name, "batch%d.bin", k);
        CK(save_dev(dir, name, items[k].out, items[k].out_size));
    }
    /* the server: compress input 0 and decompress stream 1, then poll both */
    uint64_t arena_bytes = 1ull << 30;
    void *arena = NULL;
    CK(cudaMalloc(&arena, arena_bytes));
    pc_server *srv = NULL;
    CK(pc_server_create(arena, arena_bytes, 2, &srv));
    pc_request rq[2];
    memset(rq, 0, sizeof rq);
    rq[0].kind = PC_REQ_COMPRESS;
    rq[0].dtype = in[0].dtype;
    rq[0].eb_mode = in[0].mode;
    rq[0].eb = in[0].eb;
    rq[0].input = in[0].dev;
    rq[0].n = in[0].n;
    rq[0].tag = 70;
    rq[1].kind = PC_REQ_DECOMPRESS;
    rq[1].dtype = in[1].dtype;
    rq[1].input = stream_dev[1];
    rq[1].n = in[1].n;
    rq[1].input_bytes = stream_size[1];
    rq[1].tag = 71;
    CK(pc_server_submit(srv, &rq[0]));
    CK(pc_server_submit(srv, &rq[1]));
    int done = 0;
    for (int spins = 0; done < 2 && spins < 1000; ++spins) {
        pc_completion c[2];
        uint32_t got = 0;
        CK(pc_server_poll(srv, c, 2, &got, 1));
        for (uint32_t i = 0; i < got; ++i) {
            printf("served %llu %d %d %llu\n", (unsigned long long)c[i].tag, c[i].status, c[i].kind,
                   (unsigned long long)c[i].output_bytes);
            snprintf(name, sizeof name, "served%llu.bin", (unsigned long long)c[i].tag);
            CK(save_dev(dir, name, c[i].output, c[i].output_bytes));
            CK(pc_server_release(srv, c[i].output));
            ++done;
        }
    }
    CK(pc_server_destroy(srv));
    printf("done %d\n", done);
    return done == 2 ? 0 : 1;
}
"""


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    pytest.skip("CUDA toolkit not found")


def _write_input(path, pos, mode, eb):
    dtype = 0 if pos.dtype == np.float32 else 1
    with open(path, "wb") as f:
        f.write(np.array([pos.shape[0], dtype | (mode << 8)], np.uint64).tobytes())
        f.write(np.array([eb], np.float64).tobytes())
        f.write(np.ascontiguousarray(pos).tobytes())


def test_c_program_compresses_decompresses_batches_and_serves(tmp_path, oracle_mod):
    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as b

    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    b.build()
    pc.load()
    cuda = _cuda_home()
    lib64 = next((os.path.join(cuda, d) for d in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib")
                  if os.path.exists(os.path.join(cuda, d, "libcudart.so"))), None)
    if lib64 is None:
        pytest.skip("libcudart.so not found")
    src = tmp_path / "roundtrip.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "roundtrip"
    libdir = os.path.dirname(pc.LIB_PATH)
    r = subprocess.run(["gcc", "-std=c99", "-O1", "-Wall", "-Wextra", "-Werror", "-I", INC, "-I",
                        os.path.join(cuda, "include"), str(src), "-o", str(exe), "-L", libdir,
                        "-l:" + os.path.basename(pc.LIB_PATH), "-Wl,-rpath," + libdir, "-L", lib64, "-lcudart",
                        "-Wl,-rpath," + lib64], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

    inputs = [
        (synth.cosmology(300_001, seed=21), oracle_mod.REL, 1e-3),
        (synth.fluid(200_000, seed=22), oracle_mod.ABS, 1e-4),
    ]
    assert inputs[1][0].dtype == np.float64
    paths = []
    for k, (pos, mode, eb) in enumerate(inputs):
        p = tmp_path / f"in{k}.bin"
        _write_input(p, pos, mode, eb)
        paths.append(str(p))
    run = subprocess.run([str(exe), paths[0], paths[1], str(tmp_path)], capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, run.stdout + run.stderr
    out = run.stdout.splitlines()
    assert out[-1] == "done 2"

    refs = [oracle_mod.compress(pos, mode, eb)[0] for pos, mode, eb in inputs]
    for k, (pos, mode, eb) in enumerate(inputs):
        ref = refs[k]
        assert (tmp_path / f"stream{k}.bin").read_bytes() == ref
        assert (tmp_path / f"batch{k}.bin").read_bytes() == ref
        dec = np.frombuffer((tmp_path / f"dec{k}.bin").read_bytes(), pos.dtype).reshape(-1, 3)
        assert dec.tobytes() == oracle_mod.decompress(ref).tobytes()
        n, dt, nl, _ = oracle_mod.stream_header(ref)
        info = [line for line in out if line.startswith(f"info {k} ")][0].split()
        assert [int(x) for x in info[2:7]] == [n, dt, nl, len(ref), 0]
    batch = [line.split() for line in out if line.startswith("batch ")]
    assert [(int(s), int(z)) for _, _, s, z in batch] == [(0, len(refs[0])), (0, len(refs[1]))]
    served = {int(t): (int(s), int(kind), int(z)) for _, t, s, kind, z in
              (line.split() for line in out if line.startswith("served "))}
    assert served[70] == (0, 0, len(refs[0]))
    assert served[71] == (0, 1, inputs[1][0].nbytes)
    assert (tmp_path / "served70.bin").read_bytes() == refs[0]
    assert (tmp_path / "served71.bin").read_bytes() == oracle_mod.decompress(refs[1]).tobytes()
