// Pipe-peak microbenchmarks: the roofline denominators of the integer kernels.
//
// Each kernel is a dependency-staggered stream of one inner operation of the
// semiring kernels, with eight independent accumulator chains per thread so
// issue, not latency, bounds it: step t updates acc[j] from acc[j] and
// acc[j+1] of step t-1, which keeps every operand live and varying.
//   SR_PEAK_DPX_S16X2   : acc = max(x + a, acc) per 16-bit lane (u8 product inner op)
//   SR_PEAK_U16_PAIR    : acc = max(max(x, na) + nga, acc) per lane (u16 inner op, 2 instructions)
//   SR_PEAK_LOP3        : acc |= x & m (Boolean inner op, 32 columns per instruction)
//   SR_PEAK_IADD        : acc = acc + x (plain 32-bit integer add, reference)
//   SR_PEAK_U32_PAIR    : acc = max(max(x, na) + pa, acc) on one 32-bit entry (u32 inner op, 2 instructions)

#include <algorithm>

#include "sr_common.cuh"
#include "sr_kernels.h"

namespace sr {

template <int OP>
__global__ void __launch_bounds__(256) peak_kernel(int iters, uint32_t seed, uint32_t *sink)
{
    uint32_t acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        acc[j] = (threadIdx.x * 0x9E3779B9u) ^ (seed + j * 0x01000193u);
    const uint32_t a0 = seed | 0x80008000u, a1 = seed * 3u + 0x00010001u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            uint32_t nxt[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t x = acc[(j + 1) & 7];
                if (OP == SR_PEAK_DPX_S16X2)
                    nxt[j] = __viaddmax_s16x2(x, a0, acc[j]);
                else if (OP == SR_PEAK_U16_PAIR)
                    nxt[j] = __viaddmax_u16x2(vmax_u16x2(x, a0), a1, acc[j]);
                else if (OP == SR_PEAK_U32_PAIR)
                    nxt[j] = __viaddmax_u32(max(x, a0), a1, acc[j]);
                else if (OP == SR_PEAK_LOP3)
                    nxt[j] = acc[j] | (x & acc[(j + 2) & 7]);      // one three-input LOP3
                else
                    nxt[j] = acc[j] + x;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                acc[j] = nxt[j];
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        r ^= acc[j];
    if (r == seed)          // practically never; keeps the chains alive
        sink[threadIdx.x] = r;
}

}  // namespace sr

using namespace sr;

extern "C" sr_status sr_peak_probe(int op, int iters, int blocks_per_sm, void *stream, double *ms,
                                   double *instr_per_s, double *ops_per_s)
{
    if (!ms || !instr_per_s || !ops_per_s)
        return fail(SR_EINVAL, "sr_peak_probe: NULL output");
    if (op < SR_PEAK_DPX_S16X2 || op > SR_PEAK_TC_F8)
        return fail(SR_EINVAL, "sr_peak_probe: unknown op %d", op);
    if (iters <= 0 || blocks_per_sm <= 0 || blocks_per_sm > 64)
        return fail(SR_EINVAL, "sr_peak_probe: iters > 0 and 1 <= blocks_per_sm <= 64");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (op == SR_PEAK_TC_F8)            // one CTA per SM; blocks_per_sm does not apply
        return peak_tc_f8(iters, s, ms, instr_per_s, ops_per_s);
    const int blocks = device_sm_count() * blocks_per_sm, threads = 256;
    uint32_t *sink = nullptr;
    SR_CUDA_CHECK(cudaMallocAsync(&sink, threads * sizeof(uint32_t), s));
    cudaEvent_t e0, e1;
    SR_CUDA_CHECK(cudaEventCreate(&e0));
    SR_CUDA_CHECK(cudaEventCreate(&e1));
    auto launch = [&](int n) {
        switch (op) {
        case SR_PEAK_DPX_S16X2: peak_kernel<SR_PEAK_DPX_S16X2><<<blocks, threads, 0, s>>>(n, 0x1234u, sink); break;
        case SR_PEAK_U16_PAIR: peak_kernel<SR_PEAK_U16_PAIR><<<blocks, threads, 0, s>>>(n, 0x1234u, sink); break;
        case SR_PEAK_LOP3: peak_kernel<SR_PEAK_LOP3><<<blocks, threads, 0, s>>>(n, 0x1234u, sink); break;
        case SR_PEAK_U32_PAIR: peak_kernel<SR_PEAK_U32_PAIR><<<blocks, threads, 0, s>>>(n, 0x1234u, sink); break;
        default: peak_kernel<SR_PEAK_IADD><<<blocks, threads, 0, s>>>(n, 0x1234u, sink); break;
        }
    };
    launch(std::max(1, iters / 8));                      // warm-up
    SR_CUDA_CHECK(cudaEventRecord(e0, s));
    launch(iters);
    SR_CUDA_CHECK(cudaEventRecord(e1, s));
    count_launches(2);
    SR_CUDA_CHECK(cudaEventSynchronize(e1));
    float t = 0.f;
    SR_CUDA_CHECK(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, s);
    SR_CUDA_CHECK(cudaStreamSynchronize(s));
    const double instr_per_thread = (double)iters * 16 * 8 * ((op == SR_PEAK_U16_PAIR || op == SR_PEAK_U32_PAIR) ? 2 : 1);
    const double ops_per_instr = op == SR_PEAK_DPX_S16X2 ? 2.0 : op == SR_PEAK_U16_PAIR ? 1.0
                               : op == SR_PEAK_LOP3 ? 32.0 : op == SR_PEAK_U32_PAIR ? 0.5 : 1.0;
    const double total = instr_per_thread * blocks * threads;
    *ms = t;
    *instr_per_s = total / (t * 1e-3);
    *ops_per_s = *instr_per_s * ops_per_instr;
    return SR_OK;
}
