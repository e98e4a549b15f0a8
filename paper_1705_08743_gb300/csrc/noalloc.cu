// Boolean closure by repeated squaring with a fixed, library-owned scratch
// area, for callers that cannot allocate device memory at all.
//
// bool_closure(..., SR_CLOSURE_SQUARING, ...) needs two D×D bit matrices of
// scratch, which it takes from the workspace the caller allocated through
// sr_create.  Some callers cannot make that allocation: code that runs where
// another allocator already owns all device memory (a framework's pool), a
// plugin held to a fixed memory budget, or a latency-critical loop that must
// never pay for cudaMalloc's implicit synchronisation.  This entry point
// instead uses a scratch array that is part of the library image: it exists on
// every GPU that loads the library, from load until process exit, and no call
// allocates or frees anything.
//
// Rules that follow from sharing one array:
//  - The array holds SR_NOALLOC_SCRATCH_BYTES (16 MiB); larger problems are
//    rejected with SR_EINVAL before any work is queued.
//  - Every call uses the same array, which keeps whatever the previous call
//    left in it.  Each call overwrites all scratch it later reads, so nothing
//    needs clearing, but calls that overlap on the GPU (different streams,
//    without ordering between them) race on it.
//  - The first call on a device looks up the array's device address on that
//    device (cudaGetSymbolAddress, once per device); make that first call
//    before any stream capture.
//  - The library is built without relocatable device code, so this file is a
//    module of its own, and with CUDA's default lazy module loading the module
//    (and with it the 16 MiB array) is loaded onto a device only by that first
//    address lookup.  So the first call on each device does reserve the array's
//    memory there and may synchronise the device; a caller whose allocator will
//    later own all free memory makes that first call (e.g. on a 1×1 matrix)
//    before the allocator reserves it, or sets CUDA_MODULE_LOADING=EAGER so that
//    every module is loaded when the CUDA context is created.

#include <mutex>

#include "sr_common.cuh"
#include "sr_kernels.h"
#include "sr_trace.h"

namespace sr {

constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;   // = SR_NOALLOC_SCRATCH_BYTES

// Device-side scratch.  In host code this name is only a host-side stand-in
// for the symbol, not a device address: handing it to a kernel would fault, or
// on a system where the GPU can read host memory silently use the wrong bytes.
// Host code must use the address from cudaGetSymbolAddress (see scratch_ptr).
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocScratchBytes / sizeof(uint32_t)];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
static sr_status scratch_ptr(uint32_t **out)
{
    SR_DEVICE_SLOT(dev);   // fails rather than share another device's cached address
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return cuda_fail(e, "bool_closure_squaring_noalloc: cudaGetSymbolAddress(scratch)");
        if (!p)
            return fail(SR_ECUDA, "bool_closure_squaring_noalloc: scratch has no device address");
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<uint32_t *>(g_noalloc_ptr[dev]);
    return SR_OK;
}

}  // namespace sr

using namespace sr;

extern "C" sr_status bool_closure_squaring_noalloc(void *T, int64_t ldt, int64_t D, sr_dtype dtype, void *stream)
{
    SR_TRACE("bool_closure_squaring_noalloc");
    const char *fn = "bool_closure_squaring_noalloc";
    if (dtype != SR_BOOL_W32 && dtype != SR_BOOL_W64)
        return fail(SR_EINVAL, "%s: dtype must be SR_BOOL_W32 or SR_BOOL_W64", fn);
    SR_TRY(check_dim(fn, "D", D));
    SR_TRY(check_mat(fn, "T", T, ldt, D, D, dtype));               // same bounds as bool_closure
    const int u = dtype == SR_BOOL_W64 ? 2 : 1;                  // 32-bit words per word of dtype
    const int64_t units = dtype == SR_BOOL_W64 ? (D + 63) / 64 : (D + 31) / 32;
    const int64_t rw = units * u;                                 // 32-bit words per row
    const int64_t ldw = (rw + 3) / 4 * 4;                         // scratch rows padded to 16 bytes
    const int64_t need = 2 * D * ldw * (int64_t)sizeof(uint32_t);
    if ((size_t)need > kNoallocScratchBytes)
        return fail(SR_EINVAL,
                    "%s: D = %lld needs %lld scratch bytes, more than the fixed %zu (D <= 8192 always fits)",
                    fn, (long long)D, (long long)need, kNoallocScratchBytes);

    uint32_t *M = nullptr;
    SR_TRY(scratch_ptr(&M));
    uint32_t *M2 = M + D * ldw;
    uint32_t *T32 = static_cast<uint32_t *>(T);
    const int64_t ldt32 = ldt * u;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    SR_TRY(launch_copy_rows(T32, ldt32, M, ldw, (int)D, (int)rw, s));       // M := A
    SR_TRY(launch_bool_identity_or(M, ldw, (int)D, s));                     // M := I ⊕ A
    int m = 0;
    while (((int64_t)1 << m) < (D - 1 > 1 ? D - 1 : 1)) ++m;
    auto mul32 = [&](const uint32_t *X, int64_t ldx, const uint32_t *Y, int64_t ldy, uint32_t *Z) -> sr_status {
        BoolArgs a;
        a.A = X; a.B = Y; a.C = Z;
        a.lda = ldx; a.ldb = ldy; a.ldc = ldw;
        a.R = (int)D; a.K = (int)D; a.N = (int)D;
        a.ncw = (int)rw;
        a.accumulate = 0;                                                  // Z fully overwritten
        a.skip0 = 0x7fffffff; a.skipw = 0;
        a.skip0w = 0x7fffffff; a.skipww = 0;
        const bool v = aligned16(X) && aligned16(Y) && ((ldx & 3) == 0) && ((ldy & 3) == 0);
        return launch_bool_mul(a, v, s);
    };
    for (int it = 0; it < m; ++it) {                                        // M := M ⊗ M
        SR_TRY(mul32(M, ldw, M, ldw, M2));
        uint32_t *t = M; M = M2; M2 = t;
    }
    SR_TRY(mul32(T32, ldt32, M, ldw, M2));                                 // A ⊗ (I ⊕ A)^(2^m)
    return launch_copy_rows(M2, ldw, T32, ldt32, (int)D, (int)rw, s);
}
