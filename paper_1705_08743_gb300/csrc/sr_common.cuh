// Shared device/host helpers of the semiring library (CUDA path only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/semiring.h"

namespace sr {

// ----------------------------------------------------------------- errors
// Thread-local message for sr_last_error().
void set_error(const char *fmt, ...);
sr_status fail(sr_status st, const char *fmt, ...);
sr_status cuda_fail(cudaError_t e, const char *what);

#define SR_CUDA_CHECK(call)                                  \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return ::sr::cuda_fail(_e, #call); \
    } while (0)

#define SR_TRY(call)                                         \
    do {                                                     \
        sr_status _s = (call);                               \
        if (_s != SR_OK) return _s;                          \
    } while (0)

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ----------------------------------------------------------------- lane ops
// Anti-distance entries live in 16-bit lanes, two per 32-bit register.
//
// u8 (S = 255): lanes are signed 16-bit.  The broadcast operand holds a − 255
// (in [−255, 0]) in both lanes, the other operand b (in [0, 255]), so
// b + (a − 255) = a + b − S fits a signed 16-bit lane, and
//     acc = max(b + (a − S), acc)                 (one DPX add-max per 2 lanes)
// equals acc ⊕ (a ⊗ b) = max(acc, max(a + b − S, 0)) because acc >= 0 always.
//
// u16 (S = 65535): a + b − S needs 17 bits, so the paper's saturating-subtract
// form is kept: a ⊗ b = b ⊖ (S − a) = max(b, S − a) − (S − a).  The subtraction
// is done as a wrapping 16-bit add of (a + 1) mod 2^16 = −(S − a) mod 2^16,
// fused with the max:  acc = max(max(b, na) + nga, acc),  na = S − a, nga = a + 1.
__device__ __forceinline__ uint32_t vmax_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

struct KindU8 {
    using elem = uint8_t;
    static constexpr uint32_t S = 255u;
    static constexpr int AW = 1;     // 32-bit words per broadcast A operand
    __device__ __forceinline__ static void bcast(uint32_t a, uint32_t &a0, uint32_t &a1)
    {
        a0 = __byte_perm(a + 0xFF01u, 0u, 0x1010);   // (a − 255) mod 2^16 in both lanes
        a1 = 0u;
    }
    __device__ __forceinline__ static uint32_t op(uint32_t acc, uint32_t b2, uint32_t a0, uint32_t)
    {
        return __viaddmax_s16x2(b2, a0, acc);
    }
};

struct KindU16 {
    using elem = uint16_t;
    static constexpr uint32_t S = 65535u;
    static constexpr int AW = 2;
    __device__ __forceinline__ static void bcast(uint32_t a, uint32_t &a0, uint32_t &a1)
    {
        a0 = ((~a) & 0xFFFFu) * 0x10001u;            // S − a
        a1 = ((a + 1u) & 0xFFFFu) * 0x10001u;        // −(S − a) mod 2^16
    }
    __device__ __forceinline__ static uint32_t op(uint32_t acc, uint32_t b2, uint32_t a0, uint32_t a1)
    {
        return __viaddmax_u16x2(vmax_u16x2(b2, a0), a1, acc);
    }
};

// u32 (S = 2^32 − 1): one entry per register; its kernels (antidist32.cu) carry their
// own arithmetic.  The type only names the entry for the shared closure pipeline.
struct KindU32 {
    using elem = uint32_t;
    static constexpr uint32_t S = 0xFFFFFFFFu;
};

// Pairs of u8 entries <-> one 32-bit register of two 16-bit lanes.
__device__ __forceinline__ uint32_t u8x2_lo(uint32_t w) { return __byte_perm(w, 0u, 0x4140); }  // bytes 0,1
__device__ __forceinline__ uint32_t u8x2_hi(uint32_t w) { return __byte_perm(w, 0u, 0x4342); }  // bytes 2,3
__device__ __forceinline__ uint32_t pack_u8x4(uint32_t p01, uint32_t p23) { return __byte_perm(p01, p23, 0x6420); }

}  // namespace sr
