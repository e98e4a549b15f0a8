// Fused-pass schedule of the anti-distance closure (u8, u16; 128-wide pivot blocks).
//
// Method: Section 2's Warshall loop with Section 3's Floyd ⊕/⊗, in the blocked
// three-phase order (phase 1: close the diagonal block; phase 2: its row and column
// panels; phase 3: every other block).  The stream schedules of closure.cu prepare the
// next pivot block's phases 1 and 2 on side streams beside phase 3; those small launches
// find every SM slot taken by phase-3 CTAs and start only as a wave of them retires, so
// the next block's panels land after the current phase 3 has ended and the next pass
// waits for them.  Here one launch per pivot block kb holds everything that can run
// beside phase 3 of kb, as work items in the order CTAs take them from a counter:
//   1. block kb+1's update from kb, T_{kb+1,kb+1} ⊕= T_{kb+1,kb} ⊗ T_{kb,kb+1}, as four
//      64×64 items on different SMs;
//   2. the strips: kb's update of block row and column kb+1 outside blocks kb and kb+1;
//   3. block kb+1's closure (diag128.cuh), once the four update items are done;
//   4. phase 3 of kb on every block outside block rows and columns kb and kb+1;
//   5. phase 2 of kb+1: its row panel T_{kb+1,j} ⊕= T_{kb+1,kb+1} ⊗ T_{kb+1,j} (j ≠ kb+1)
//      and column panel T_{i,kb+1} ⊕= T_{i,kb+1} ⊗ T_{kb+1,kb+1} (i ≠ kb+1), in place, once
//      the closure and every strip are done.
// Items 1, 2 and 4 are independent: 1 and 3 write block (kb+1, kb+1), 2 the rest of row
// and column kb+1, 4 the blocks outside rows and columns kb and kb+1; all of them read
// only panel kb (final since the previous launch) and what they write.  Items 3 and 5
// wait on counters (release/acquire order, operands read through L2) that items taken
// earlier by running CTAs raise, so each wait ends; it is still bounded (the context's
// spin limit: a wait that gives up sets the context's status word and skips its item,
// sr_stream_status reports SR_ETIMEOUT).  The launch of kb+1 follows on the same stream,
// with block kb+1 closed and its panels done; a launch with kb = -1 closes block 0 and
// makes its panels.  Consecutive launches use programmatic dependent launch: the next
// one's CTAs take the slots the current one's last CTAs leave and wait in hardware until
// it has completed, so no launch gap separates the passes.
//
// GB300, against the stream schedule: u8 D = 4096 2.48 / 2.64 ms, u16 D = 4096 4.67 /
// 4.73 ms; slower at u8 D = 2048 (1.22 / 0.82), 3584 (2.12 / 1.96) and 6144 (7.82 /
// 7.29), where the stream schedule's peer stream or a better-filled last wave wins.  The
// autotuner times it beside the other schedules (SR_TUNE_FUSED).

#include <algorithm>

#include "antidist_tile.cuh"
#include "diag128.cuh"
#include "sr_common.cuh"
#include "sr_kernels.h"
#include "sr_trace.h"

namespace sr {
namespace {

constexpr int FB = 128;                  // pivot block and product tile side
constexpr int FQ = 64;                   // tile side of the diagonal block's update (four items)
constexpr int FNONE = 0x7fffffff;        // no excluded range
constexpr int kCtrInts = 4;              // per launch: [0] next item, [1] phase 1 done, [2] strips done,
                                         // [3] update quarters done

struct FusedArgs {
    void *T;
    int64_t ldt;
    int D, nb, kb;              // order, 128-wide blocks, this launch's pivot block (-1: block 0's phases 1-2)
    int *ctr;                   // this launch's kCtrInts counters, zeroed before the launch
    int *status;                // the context's status words: [0] code, [1] where
    uint32_t limit;             // tries per wait
};

// items of the launch for pivot block kb (geometry shared by host and device)
struct FusedShape {
    int k0, bw, k1, bwn, ex;    // block kb at [k0, k0+bw), block kb+1 at [k1, k1+bwn); ex = bw + bwn
    int tn, tp;                 // tiles per side outside rows/columns kb, kb+1; tiles of each panel of kb+1
    int n_upd, n_strip, n_piv, n_p3, n_panel;
    __host__ __device__ FusedShape(int D, int nb, int kb)
    {
        const bool next = kb + 1 < nb;
        k0 = kb < 0 ? 0 : kb * FB;
        bw = kb < 0 ? 0 : (D - k0 < FB ? D - k0 : FB);
        k1 = kb < 0 ? 0 : k0 + bw;
        bwn = next ? (D - k1 < FB ? D - k1 : FB) : 0;
        ex = bw + bwn;
        tn = kb < 0 ? 0 : (D - ex + FB - 1) / FB;
        tp = next ? (D - bwn + FB - 1) / FB : 0;
        const int tq = (bwn + FQ - 1) / FQ;               // quarter tiles per side of block kb+1
        n_upd = next && kb >= 0 ? tq * tq : 0;
        n_piv = next ? 1 : 0;
        n_strip = next ? 2 * tn : 0;
        n_p3 = tn * tn;
        n_panel = 2 * tp;
    }
    __host__ __device__ int items() const { return n_upd + n_strip + n_piv + n_p3 + n_panel; }
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits (bounded) until every counter c[i] >= v[i]; the CTA then learns whether
// the wait succeeded.  A wait that gives up sets the status word (code 1, where 4).
__device__ __forceinline__ bool wait_counts(const FusedArgs &a, const int *c0, int v0, const int *c1, int v1)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        uint32_t tries = 0;
        while (ld_acquire_gpu(c0) < v0 || ld_acquire_gpu(c1) < v1) {
            if (tries++ >= a.limit) {                     // limit 0: give up at the first unmet check
                ok = 0;
                if (a.status) {
                    atomicExch(a.status + 1, 4);          // where: the fused-pass closure
                    atomicExch(a.status, 1);
                }
                break;
            }
            __nanosleep(128);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class KD, bool VEC>
__global__ void __launch_bounds__(MulCfg<KD, FB, FB, 32, 8, 16>::THREADS, MulCfg<KD, FB, FB, 32, 8, 16>::MIN_BLOCKS)
closure_fused_kernel(FusedArgs a)
{
    using E = typename KD::elem;
    __shared__ int s_item;
    extern __shared__ __align__(16) uint32_t smem[];
    E *T = static_cast<E *>(a.T);
    const int64_t ld = a.ldt;
    const FusedShape f(a.D, a.nb, a.kb);

    // programmatic dependent launch: the next launch may start its CTAs once every CTA of
    // this one has started; each CTA waits here until the previous launch has completed
    // and its writes are visible (a no-op when launched without the attribute)
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");

    if (threadIdx.x == 0) {
        s_item = atomicAdd(&a.ctr[0], 1);
    }
    __syncthreads();
    int it = s_item;

    MulArgs p;
    p.lda = p.ldb = p.ldc = ld;
    p.accumulate = 1;
    p.rskip0 = p.cskip0 = FNONE;
    p.rskipw = p.cskipw = 0;
    p.skip_tile = -1;
    p.group_m = 0;
    p.split = 0;

    if (it < f.n_upd) {                                   // 1a. block kb+1's update from kb, a quarter
        p.A = T + (int64_t)f.k1 * ld + f.k0;
        p.B = T + (int64_t)f.k0 * ld + f.k1;
        p.C = T + (int64_t)f.k1 * ld + f.k1;
        p.R = f.bwn; p.N = f.bwn; p.K = f.bw;
        mul_tiles<KD, FQ, FQ, 32, 4, 8, VEC>(p, it, 1 << 30);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&a.ctr[3], 1);
        }
        return;
    }
    it -= f.n_upd;
    if (it >= f.n_strip && it < f.n_strip + f.n_piv) {    // 1b. block kb+1's closure, after its update
        if (!wait_counts(a, &a.ctr[3], f.n_upd, &a.ctr[3], f.n_upd))
            return;
        diag::close_diag128<KD, 0>(T, ld, a.D, f.k1, smem);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_gpu(&a.ctr[1], 1);
        }
        return;
    }
    // items 2, 4 and 5 share one call of the tile routine (one copy of its unrolled k-loop
    // for the instruction cache); its loads go through L2, which item 5 needs
    const bool strip = it < f.n_strip;
    if (strip) {                                          // 2. kb's update of row / column kb+1
        if (it < f.tn) {
            p.A = T + (int64_t)f.k1 * ld + f.k0;
            p.B = T + (int64_t)f.k0 * ld;
            p.C = T + (int64_t)f.k1 * ld;
            p.R = f.bwn; p.N = a.D - f.ex; p.K = f.bw;
            p.cskip0 = f.k0; p.cskipw = f.ex;
        } else {
            it -= f.tn;
            p.A = T + f.k0;
            p.B = T + (int64_t)f.k0 * ld + f.k1;
            p.C = T + f.k1;
            p.R = a.D - f.ex; p.N = f.bwn; p.K = f.bw;
            p.rskip0 = f.k0; p.rskipw = f.ex;
        }
    } else {
        it -= f.n_strip + f.n_piv;
        if (it < f.n_p3) {                                // 4. phase 3 of kb
            p.A = T + f.k0;
            p.B = T + (int64_t)f.k0 * ld;
            p.C = T;
            p.R = a.D - f.ex; p.N = a.D - f.ex; p.K = f.bw;
            p.rskip0 = p.cskip0 = f.k0;
            p.rskipw = p.cskipw = f.ex;
        } else {
            it -= f.n_p3;
            if (it >= f.n_panel)
                return;
            // 5. phase 2 of kb+1, once block kb+1 is closed and the strips are done
            if (!wait_counts(a, &a.ctr[1], 1, &a.ctr[2], f.n_strip))
                return;
            if (it < f.tp) {                              // row panel of kb+1, in place
                p.A = T + (int64_t)f.k1 * ld + f.k1;
                p.B = p.C = T + (int64_t)f.k1 * ld;
                p.R = f.bwn; p.N = a.D - f.bwn; p.K = f.bwn;
                p.cskip0 = f.k1; p.cskipw = f.bwn;
            } else {                                      // column panel of kb+1, in place
                it -= f.tp;
                p.A = p.C = T + f.k1;
                p.B = T + (int64_t)f.k1 * ld + f.k1;
                p.R = a.D - f.bwn; p.N = f.bwn; p.K = f.bwn;
                p.rskip0 = f.k1; p.rskipw = f.bwn;
            }
        }
    }
    mul_tiles<KD, FB, FB, 32, 8, 16, VEC, true>(p, it, 1 << 30);
    if (strip) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&a.ctr[2], 1);
        }
    }
}

template <class KD>
sr_status launch_fused(void *T, int64_t ldt, int D, void *ws, size_t ws_bytes, int *status, int spin_limit,
                       cudaStream_t s)
{
    using Cfg = MulCfg<KD, FB, FB, 32, 8, 16>;
    constexpr size_t SMEM = std::max(Cfg::SMEM, diag::kDiagSmem);
    const int nb = (D + FB - 1) / FB;
    const size_t need = closure_fused_workspace(D);
    if (!ws || ws_bytes < need)
        return fail(SR_EINVAL, "fused closure: workspace of %zu bytes needed", need);
    auto kern = closure_fused_kernel<KD, true>;
    static bool attr[kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
        attr[dev] = true;
    }
    int *ctr = static_cast<int *>(ws);
    SR_CUDA_CHECK(cudaMemsetAsync(ctr, 0, need, s));
    for (int kb = -1; kb < nb; ++kb) {
        SR_TRACE_BLOCK("antidist_closure.block", kb);
        const FusedShape f(D, nb, kb);
        const int n = f.items();
        if (n <= 0)
            continue;
        FusedArgs a;
        a.T = T; a.ldt = ldt; a.D = D; a.nb = nb; a.kb = kb;
        a.ctr = ctr + (size_t)(kb + 1) * kCtrInts;
        a.status = status;
        a.limit = spin_limit > 0 ? (uint32_t)spin_limit : 0u;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)n);
        lc.blockDim = dim3(Cfg::THREADS);
        lc.dynamicSmemBytes = SMEM;
        lc.stream = s;
        cudaLaunchAttribute la[1];
        la[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        la[0].val.programmaticStreamSerializationAllowed = kb >= 0 ? 1 : 0;   // after another fused launch
        lc.attrs = la;
        lc.numAttrs = 1;
        SR_CUDA_CHECK(cudaLaunchKernelEx(&lc, kern, a));
        count_launches();
    }
    return SR_OK;
}

}  // namespace

size_t closure_fused_workspace(int64_t D)
{
    if (D <= 0 || D > kPersistentMaxD)
        return 0;
    const int64_t nb = (D + FB - 1) / FB;
    return (size_t)(nb + 1) * kCtrInts * sizeof(int);
}

sr_status launch_antidist_closure_fused(void *T, int64_t ldt, int D, sr_dtype dt, void *ws, size_t ws_bytes,
                                        int *status, int spin_limit, cudaStream_t s)
{
    if (D <= 0)
        return SR_OK;
    if (dt == SR_U8)
        return launch_fused<KindU8>(T, ldt, D, ws, ws_bytes, status, spin_limit, s);
    if (dt == SR_U16)
        return launch_fused<KindU16>(T, ldt, D, ws, ws_bytes, status, spin_limit, s);
    return fail(SR_EINVAL, "fused closure: dtype must be SR_U8 or SR_U16");
}

}  // namespace sr
