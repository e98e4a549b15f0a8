/* A plain C consumer of libsemiring.so: include/semiring.h and the CUDA runtime, no
 * Python.  Reads an order-D u8 anti-distance matrix from a file, copies it to the
 * device, closes it with antidist_closure (Section 2 Warshall / Section 3 Floyd) on
 * a stream of its own, with and without a context holding the workspace
 * sr_workspace_query asks for, copies both results back and writes the first.
 * Exit status 0 only if every call succeeded and both results agree.
 *
 *   closure_c <D> <input file, D*D bytes> <output file> */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "semiring.h"

static int check_cuda(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
        return 1;
    }
    return 0;
}

static int check_sr(sr_status s, const char *what)
{
    if (s != SR_OK) {
        fprintf(stderr, "%s: status %d: %s\n", what, (int)s, sr_last_error());
        return 1;
    }
    return 0;
}

int main(int argc, char **argv)
{
    if (argc != 4) {
        fprintf(stderr, "usage: %s D input output\n", argv[0]);
        return 2;
    }
    const long long D = atoll(argv[1]);
    const size_t n = (size_t)(D * D);
    unsigned char *h = (unsigned char *)malloc(n), *h2 = (unsigned char *)malloc(n);
    if (!h || !h2) return 2;
    FILE *f = fopen(argv[2], "rb");
    if (!f || fread(h, 1, n, f) != n) {
        fprintf(stderr, "cannot read %s\n", argv[2]);
        return 2;
    }
    fclose(f);

    void *T = NULL, *T2 = NULL;
    cudaStream_t s;
    if (check_cuda(cudaStreamCreate(&s), "cudaStreamCreate")) return 1;
    if (check_cuda(cudaMalloc(&T, n), "cudaMalloc") || check_cuda(cudaMalloc(&T2, n), "cudaMalloc")) return 1;
    if (check_cuda(cudaMemcpyAsync(T, h, n, cudaMemcpyHostToDevice, s), "copy in")) return 1;
    if (check_cuda(cudaMemcpyAsync(T2, h, n, cudaMemcpyHostToDevice, s), "copy in")) return 1;

    /* no context: the stream schedule */
    if (check_sr(antidist_closure(NULL, T, D, D, SR_U8, (void *)s), "antidist_closure")) return 1;

    /* a context with the workspace the library asks for (the persistent schedule) */
    size_t ws = 0;
    if (check_sr(sr_workspace_query(SR_OP_ANTIDIST_CLOSURE, SR_U8, D, 0, &ws), "sr_workspace_query")) return 1;
    sr_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.workspace_bytes = ws;
    sr_ctx *ctx = NULL;
    if (check_sr(sr_create(&ctx, &cfg), "sr_create")) return 1;
    if (check_sr(antidist_closure(ctx, T2, D, D, SR_U8, (void *)s), "antidist_closure (ctx)")) return 1;
    if (check_sr(sr_stream_status(ctx, (void *)s), "sr_stream_status")) return 1;

    if (check_cuda(cudaMemcpyAsync(h, T, n, cudaMemcpyDeviceToHost, s), "copy out")) return 1;
    if (check_cuda(cudaMemcpyAsync(h2, T2, n, cudaMemcpyDeviceToHost, s), "copy out")) return 1;
    if (check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize")) return 1;
    sr_destroy(ctx);
    cudaFree(T);
    cudaFree(T2);
    cudaStreamDestroy(s);

    if (memcmp(h, h2, n) != 0) {
        fprintf(stderr, "the two schedules disagree\n");
        return 1;
    }
    f = fopen(argv[3], "wb");
    if (!f || fwrite(h, 1, n, f) != n) return 2;
    fclose(f);
    free(h);
    free(h2);
    printf("ok %s\n", sr_version());
    return 0;
}
