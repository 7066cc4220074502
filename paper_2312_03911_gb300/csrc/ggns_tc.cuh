// ggns_tc.cuh -- the dense contraction y = P v of the correlated-Gaussian and
// dense-mixture likelihoods on the fifth-generation tensor cores (tcgen05).
//
// One CTA steps 16 walkers (one per warp).  Each step, the walkers' vectors v
// (x - mu, or x for the mixture) are split into TF32 pairs v = v_hi + v_lo and
// written to shared memory as the B operand (N = 16 walkers, K-major core
// matrices).  The precision matrix, pre-split into P_hi + P_lo and pre-laid-out
// in core-matrix order when the context is created, streams from global memory through a ring
// of shared-memory stages (one K-step of 8 columns of P per stage, for every
// 128-row M-tile) with 1-D bulk copies completing on mbarriers.  One thread
// issues, per K-step and M-tile, the three MMAs of the 3xTF32 product
// P_hi v_hi + P_hi v_lo + P_lo v_hi (M = 128, N = 16, K = 8, FP32 accumulation
// in tensor memory), and refills each stage once its MMAs have completed.  The
// accumulators, Y^T[d_pad][16] (P is symmetric, so Y^T = P V^T), are read back
// with tcgen05.ld and handed to the walkers through shared memory.  The split
// keeps the product at FP32 accuracy (the neglected P_lo v_lo is 2^-22 relative).
//
// Every wait is bounded (2 s): a wait that gives up sets the CTA's failure flag,
// the run's status NS_ERR_TIMEOUT, and the kernel winds down, waiting (again
// bounded) for its MMAs and copies in flight and freeing its tensor memory.
#pragma once

#include "ggns_internal.cuh"

namespace ggns {
namespace tc {

constexpr int WALKERS = 16;                    // N of every MMA: one walker per warp of a 512-thread CTA
constexpr int STAGES = 3;                      // shared-memory stages of P in flight
constexpr uint64_t WAIT_NS = 2000000000ull;    // a wait gives up after 2 s

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `bar` with the given parity to complete; false if it did not
// within WAIT_NS nanoseconds.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > WAIT_NS) return false;
    }
}

// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16),
// completing its bytes on `bar`.
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, K-major core matrices (8 rows x 16 bytes,
// contiguous); lbo = bytes between core matrices along K, sbo = bytes between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;  // descriptor version of the fifth-generation tensor cores
    return d;
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every MMA this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 16 consecutive 32-bit columns of the warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_load16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Layout of the tensor-core state in dynamic shared memory (bytes from a 1024-aligned base).
struct Plan {
    int mt, ks;              // 128-row M-tiles and 8-column K-steps of d_pad
    uint32_t stage_bytes;    // one K-step of P_hi and P_lo for every M-tile
    uint32_t v_off, stage_off, bar_off, total;
};

__host__ __device__ inline Plan plan(int d_pad)
{
    Plan p;
    p.mt = d_pad / 128;
    p.ks = d_pad / 8;
    p.stage_bytes = static_cast<uint32_t>(2 * p.mt * 4096);
    p.v_off = 0;                                            // V_hi then V_lo: 2 x ks x 512 bytes
    p.stage_off = p.v_off + static_cast<uint32_t>(2 * p.ks * 512);
    p.bar_off = p.stage_off + STAGES * p.stage_bytes;       // full[S], empty[S], done, tmem base
    p.total = p.bar_off + (2 * STAGES + 1) * 8 + 16;
    return p;
}

// Floats of the pre-laid-out P of a run: ks K-steps x (P_hi, P_lo) x mt tiles x 1024.
__host__ __device__ inline long ptc_floats(int d_pad) { return 2l * d_pad * d_pad; }

// Per-CTA state (shared-memory pointers, tensor-memory base, pipeline counters).
struct State {
    float *vhi, *vlo;     // B operand (Y^T aliases vhi after the MMAs)
    char *stages;
    uint64_t *full, *empty, *done;
    uint32_t *tmem_slot;
    uint32_t tmem;        // tensor-memory base address (lane 0, first column)
    uint32_t ncols;       // allocated columns
    const float *ptc;     // pre-laid-out P of the run (global)
    int mt, ks;
    uint32_t stage_bytes;
    long g;               // K-steps consumed so far (thread 0 only)
    uint32_t done_phase;  // parity of the next completion of `done` (every thread)
    int *fail;            // shared failure flag
};

// CTA set-up: barriers, tensor memory, the first STAGES K-steps of P.  Every thread
// calls it; `base` is 1024-byte aligned dynamic shared memory of plan(d_pad).total bytes.
__device__ inline void setup(State &T, char *base, const float *ptc, int d_pad, int *fail_flag)
{
    const Plan pl = plan(d_pad);
    T.vhi = reinterpret_cast<float *>(base + pl.v_off);
    T.vlo = reinterpret_cast<float *>(base + pl.v_off + pl.ks * 512);
    T.stages = base + pl.stage_off;
    T.full = reinterpret_cast<uint64_t *>(base + pl.bar_off);
    T.empty = T.full + STAGES;
    T.done = T.empty + STAGES;
    T.tmem_slot = reinterpret_cast<uint32_t *>(T.done + 1);
    T.ptc = ptc;
    T.mt = pl.mt;
    T.ks = pl.ks;
    T.stage_bytes = pl.stage_bytes;
    T.g = 0;
    T.done_phase = 0;
    T.fail = fail_flag;
    T.ncols = (pl.mt * WALKERS <= 32) ? 32u : static_cast<uint32_t>(pl.mt * WALKERS);  // a power of two
    if (threadIdx.x == 0) {
        *fail_flag = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(T.full + s, 1);
            mbar_init(T.empty + s, 1);
        }
        mbar_init(T.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(T.tmem_slot)),
                     "r"(T.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    T.tmem = *T.tmem_slot;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            const int j = s % T.ks;
            mbar_expect_tx(T.full + s, T.stage_bytes);
            bulk_copy(T.stages + (size_t)s * T.stage_bytes, T.ptc + (size_t)j * (T.stage_bytes / 4), T.stage_bytes,
                      T.full + s);
        }
    }
}

// CTA wind-down: the copies still in flight (the prefetched stages) land, then the
// tensor memory is freed.  Every thread calls it.
__device__ inline void teardown(State &T)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        // every MMA this thread issued has completed before the tensor memory is freed
        mma_commit(T.done);
        if (!mbar_wait(T.done, T.done_phase)) *T.fail = 1;
        for (int i = 0; i < STAGES; ++i) {
            const long g = T.g + i;
            if (!mbar_wait(T.full + (g % STAGES), static_cast<uint32_t>((g / STAGES) & 1))) *T.fail = 1;
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(T.tmem), "r"(T.ncols) : "memory");
}

// Thread 0: the MMAs of one contraction, refilling each stage of P once its MMAs are
// done (the refill of the stage consumed by K-step j - 1 is issued after the MMAs of
// K-step j, so the tensor pipe always has work queued while the thread waits).
__device__ inline void issue(State &T)
{
    const uint32_t idesc = instr_desc_tf32(128, WALKERS);
    const uint32_t vhi = smem_addr(T.vhi), vlo = smem_addr(T.vlo), st0 = smem_addr(T.stages);
    const uint32_t tile_bytes = 4096u, lo_off = static_cast<uint32_t>(T.mt) * 4096u;
    const long g0 = T.g;
    bool ok = true;
    for (int j = 0; j < T.ks && ok; ++j) {
        const long g = g0 + j;
        const int s = static_cast<int>(g % STAGES);
        if (!mbar_wait(T.full + s, static_cast<uint32_t>((g / STAGES) & 1))) {
            ok = false;
            break;
        }
        fence_after_sync();
        const uint32_t sa = st0 + static_cast<uint32_t>(s) * T.stage_bytes;
        const uint64_t bh = smem_desc(vhi + 512u * j, 128, 256), bl = smem_desc(vlo + 512u * j, 128, 256);
        for (int m = 0; m < T.mt; ++m) {
            const uint64_t ah = smem_desc(sa + m * tile_bytes, 128, 256);
            const uint64_t al = smem_desc(sa + lo_off + m * tile_bytes, 128, 256);
            const uint32_t d = T.tmem + static_cast<uint32_t>(m * WALKERS);
            mma_tf32(d, ah, bh, idesc, j > 0 ? 1u : 0u);
            mma_tf32(d, ah, bl, idesc, 1u);
            mma_tf32(d, al, bh, idesc, 1u);
        }
        mma_commit(T.empty + s);
        if (j >= 1) {
            const long gp = g - 1;
            const int sp = static_cast<int>(gp % STAGES);
            if (!mbar_wait(T.empty + sp, static_cast<uint32_t>((gp / STAGES) & 1))) {
                ok = false;
                break;
            }
            const int jn = static_cast<int>((gp + STAGES) % T.ks);
            mbar_expect_tx(T.full + sp, T.stage_bytes);
            bulk_copy(T.stages + (size_t)sp * T.stage_bytes, T.ptc + (size_t)jn * (T.stage_bytes / 4),
                      T.stage_bytes, T.full + sp);
        }
    }
    if (ok) {
        const long gp = g0 + T.ks - 1;
        const int sp = static_cast<int>(gp % STAGES);
        if (mbar_wait(T.empty + sp, static_cast<uint32_t>((gp / STAGES) & 1))) {
            const int jn = static_cast<int>((gp + STAGES) % T.ks);
            mbar_expect_tx(T.full + sp, T.stage_bytes);
            bulk_copy(T.stages + (size_t)sp * T.stage_bytes, T.ptc + (size_t)jn * (T.stage_bytes / 4),
                      T.stage_bytes, T.full + sp);
        } else {
            ok = false;
        }
    }
    if (!ok) {
        *T.fail = 1;
        return;
    }
    T.g = g0 + T.ks;
    mma_commit(T.done);
}

// y = P v for the 16 walkers of the CTA (lane l of warp n holds components c0 .. c0+E-1
// of walker n).  Every thread of the CTA calls it (barriers inside).  Returns false if
// a wait gave up (y is then undefined).
template <int E>
__device__ inline bool contract(State &T, const float (&v)[E], int c0, int d_pad, float (&y)[E])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // B operand: element (walker n, column c) at K-step c / 8, core matrix ((n / 8), (c % 8) / 4)
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = c0 + e, j = c >> 3, kk = c & 7;
        const int off = j * 128 + (warp >> 3) * 64 + (kk >> 2) * 32 + (warp & 7) * 4 + (kk & 3);  // floats
        const uint32_t hi = to_tf32(v[e]);
        const uint32_t lo = to_tf32(v[e] - __uint_as_float(hi));
        T.vhi[off] = __uint_as_float(hi);
        T.vlo[off] = __uint_as_float(lo);
    }
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0 && !*T.fail) {
        fence_after_sync();
        issue(T);
    }
    // every thread: the accumulators are complete
    const bool ok = mbar_wait(T.done, T.done_phase);
    T.done_phase ^= 1u;
    fence_after_sync();
    float *ybuf = T.vhi;  // Y^T[walker][d_pad] over the B operand, free once the MMAs are done
    if (ok && warp < 4 * T.mt) {
        const int m = warp >> 2, q = warp & 3;
        float acc[16];
        tmem_load16(T.tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(m * WALKERS), acc);
        const int row = m * 128 + 32 * q + lane;
#pragma unroll
        for (int n = 0; n < WALKERS; ++n) ybuf[n * d_pad + row] = acc[n];
    }
    fence_before_sync();
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) y[e] = ybuf[warp * d_pad + c0 + e];
    __syncthreads();  // ybuf is the next contraction's B operand
    return ok && !*T.fail;
}

}  // namespace tc
}  // namespace ggns
