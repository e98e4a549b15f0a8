// Entrywise operations (the Conclusion's table) and the reflexive closure.
//
//   op AND:  a & b = min(a, b)        op OR:  a | b = max(a, b)
//   op XOR:  a ^ b = |a − b|          op NOT: ~a = S − a
// On Boolean bit matrices these are the word-wise AND, OR, XOR and NOT, with pad
// bits written 0.  The reflexive closure adds the identity: T := I ⊕ T sets the
// diagonal to S (anti-distance: distance 0) or to 1 (Boolean) (Introduction: the
// reflexive and non-reflexive closures differ by I).

#include <algorithm>

#include "sr_common.cuh"
#include "sr_kernels.h"

namespace sr {

template <class E>
__device__ __forceinline__ uint32_t ew(int op, uint32_t a, uint32_t b, uint32_t S)
{
    switch (op) {
    case SR_EW_AND: return a < b ? a : b;
    case SR_EW_OR: return a > b ? a : b;
    case SR_EW_XOR: return a > b ? a - b : b - a;
    default: return S - a;
    }
}

template <class E>
__global__ void entrywise_kernel(int op, const E *A, int64_t lda, const E *B, int64_t ldb, E *C, int64_t ldc,
                                 int R, int N, uint32_t S)
{
    const int64_t total = (int64_t)R * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / N, c = t % N;
        const uint32_t a = A[r * lda + c];
        const uint32_t b = B ? (uint32_t)B[r * ldb + c] : 0u;
        C[r * ldc + c] = (E)ew<E>(op, a, b, S);
    }
}

// Boolean words: rw 32-bit words per row, nbits valid bits
__global__ void entrywise_bits_kernel(int op, const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb,
                                      uint32_t *C, int64_t ldc, int R, int rw, int nbits)
{
    const int64_t total = (int64_t)R * rw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / rw;
        const int w = (int)(t % rw);
        const uint32_t a = A[r * lda + w], b = B ? B[r * ldb + w] : 0u;
        uint32_t v;
        switch (op) {
        case SR_EW_AND: v = a & b; break;
        case SR_EW_OR: v = a | b; break;
        case SR_EW_XOR: v = a ^ b; break;
        default: v = ~a; break;
        }
        const int lo = 32 * w;
        const uint32_t mask = lo + 32 <= nbits ? 0xFFFFFFFFu : (lo >= nbits ? 0u : (1u << (nbits - lo)) - 1u);
        C[r * ldc + w] = v & mask;
    }
}

template <class E>
__global__ void reflexive_kernel(E *T, int64_t ldt, int D, E one)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D; i += gridDim.x * blockDim.x)
        T[(int64_t)i * ldt + i] = one;
}

__global__ void reflexive_bits_kernel(uint32_t *T, int64_t ldt, int D)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D; i += gridDim.x * blockDim.x)
        T[(int64_t)i * ldt + i / 32] |= 1u << (i % 32);
}

static int blocks_for(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count() * 16));
}

sr_status launch_entrywise(int op, const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc,
                           int R, int N, sr_dtype dt, cudaStream_t s)
{
    if (dt == SR_U8)
        entrywise_kernel<uint8_t><<<blocks_for((int64_t)R * N), 256, 0, s>>>(
            op, static_cast<const uint8_t *>(A), lda, static_cast<const uint8_t *>(B), ldb, static_cast<uint8_t *>(C),
            ldc, R, N, 255u);
    else if (dt == SR_U16)
        entrywise_kernel<uint16_t><<<blocks_for((int64_t)R * N), 256, 0, s>>>(
            op, static_cast<const uint16_t *>(A), lda, static_cast<const uint16_t *>(B), ldb,
            static_cast<uint16_t *>(C), ldc, R, N, 65535u);
    else if (dt == SR_U32)
        entrywise_kernel<uint32_t><<<blocks_for((int64_t)R * N), 256, 0, s>>>(
            op, static_cast<const uint32_t *>(A), lda, static_cast<const uint32_t *>(B), ldb,
            static_cast<uint32_t *>(C), ldc, R, N, 0xFFFFFFFFu);
    else {
        const int u = dt == SR_BOOL_W64 ? 2 : 1;
        const int rw = dt == SR_BOOL_W64 ? 2 * ((N + 63) / 64) : (N + 31) / 32;
        entrywise_bits_kernel<<<blocks_for((int64_t)R * rw), 256, 0, s>>>(
            op, static_cast<const uint32_t *>(A), lda * u, static_cast<const uint32_t *>(B), ldb * u,
            static_cast<uint32_t *>(C), ldc * u, R, rw, N);
    }
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_reflexive(void *T, int64_t ldt, int D, sr_dtype dt, cudaStream_t s)
{
    if (dt == SR_U8)
        reflexive_kernel<uint8_t><<<blocks_for(D), 256, 0, s>>>(static_cast<uint8_t *>(T), ldt, D, (uint8_t)255);
    else if (dt == SR_U16)
        reflexive_kernel<uint16_t><<<blocks_for(D), 256, 0, s>>>(static_cast<uint16_t *>(T), ldt, D, (uint16_t)65535);
    else if (dt == SR_U32)
        reflexive_kernel<uint32_t><<<blocks_for(D), 256, 0, s>>>(static_cast<uint32_t *>(T), ldt, D, 0xFFFFFFFFu);
    else
        reflexive_bits_kernel<<<blocks_for(D), 256, 0, s>>>(static_cast<uint32_t *>(T),
                                                            ldt * (dt == SR_BOOL_W64 ? 2 : 1), D);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

}  // namespace sr
