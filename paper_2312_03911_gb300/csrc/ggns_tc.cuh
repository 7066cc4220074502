// ggns_tc.cuh -- the dense contraction y = P v of the correlated-Gaussian and
// dense-mixture likelihoods on the fifth-generation tensor cores (tcgen05).
//
// One CTA steps 16 walkers (one per warp).  Each step, the walkers' vectors v
// (x - mu, or x for the mixture) are scaled by a power of two s_v and split into
// FP16 pairs s_v v = V1 + 2^-11 V2, written to shared memory as the B operand
// (N = 16 walkers, K-major core matrices).  The precision matrix, scaled by a power
// of two s_p and split the same way (s_p P = P1 + 2^-11 P2) and pre-laid-out in
// core-matrix order when the context is created, streams from global memory through
// a ring of STAGES shared-memory stages of 32 KB (a stage holds P1 and P2 of one
// K-step of 16 columns for every 128-row M-tile, or of several K-steps when d_pad is
// small).  V1 and V2 form one B operand of 32 rows per K-step, so lane 0 of warp 0
// issues, per K-step and 128-row tile, two MMAs (kind::f16, K = 16, FP32 accumulation
// in tensor memory): P1 [V1 | V2] with N = 32 and P2 V1 with N = 16, each into an
// accumulator of its own (an MMA never waits for the one issued just before it; at
// these widths an MMA costs about the same time whatever its N, so the merge saves a
// third of the tensor time), and commits each stage's MMAs to that stage's `empty`
// barrier.  The read-back forms
//     y = (P1 V1 + 2^-11 (P1 V2 + P2 V1)) / (s_p s_v),
// whose neglected term 2^-22 P2 V2 and the split's rounding leave y within about
// 2^-22 of |P| |v| (each factor carries 22 significant bits; the scales keep every
// FP16 value in the normal range of its own magnitude).  Against a split into TF32
// pairs this halves the bytes of P streamed per step and the B operand in shared
// memory, and it runs at the FP16 rate.
// Stage s is refilled by lane 0 of warp 1 + s with a 1-D bulk copy once the MMAs
// that read it are done: an SM completes the bulk copies of one issuing warp one
// after another, so the copies of several warps are what keeps enough bytes in
// flight to cover the latency of the L2.  The accumulators, Y^T[d_pad][16] (P is
// symmetric, so Y^T = P V^T), are read back with tcgen05.ld and handed to the
// walkers through shared memory.
//
// Every wait is bounded (2 s): a wait that gives up sets the CTA's failure flag,
// the run's status NS_ERR_TIMEOUT, and the kernel winds down, waiting (again
// bounded) for its MMAs and copies in flight and freeing its tensor memory.
#pragma once

#include <cuda_fp16.h>

#include "ggns_internal.cuh"

namespace ggns {
namespace tc {

constexpr int WALKERS = 16;                    // N of every MMA: one walker per warp of a 512-thread CTA
constexpr int STAGES = 4;                      // shared-memory stages of P (one producer warp each)
constexpr uint32_t STAGE_BYTES = 32768;        // bytes of one stage (eight of 16 KB: 1.5x slower)
constexpr uint64_t WAIT_NS = 2000000000ull;    // a wait gives up after 2 s

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Two FP16 values in one 32-bit word (lo at the lower address).
__device__ __forceinline__ uint32_t pack_half2(float lo, float hi)
{
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
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

// Non-blocking test of the phase of `bar` with the given parity.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_wait, polling without suspending the thread: for the single lanes that feed
// the tensor cores, whose other warp-mates wait at a warp barrier.
__device__ __forceinline__ bool mbar_poll(uint64_t *bar, uint32_t parity)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (global_ns() - t0 > WAIT_NS) return false;
    }
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

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B FP16 (format 0 in
// bits 7-9 and 10-12), both K-major, dense, N / 8 in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc_f16(int M, int N)
{
    return (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

// (No memory clobber: the operands were published by the barriers and fences before
// the MMAs; keeping shared-memory reads of the issuing loop in registers across the
// MMAs is what lets one lane issue them back to back.)
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
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

// A warp keeps E floats per lane (E = 4, 8 or 16) in its lanes of tensor memory at
// column `col` (32x32b shape: lane l of the warp is tensor-memory lane 32 (warp % 4) + l),
// or reads them back.
template <int E>
__device__ __forceinline__ void tmem_store(uint32_t taddr, const float (&v)[E])
{
    static_assert(E == 4 || E == 8 || E == 16, "4, 8 or 16 columns");
    uint32_t r[E];
#pragma unroll
    for (int i = 0; i < E; ++i) r[i] = __float_as_uint(v[i]);
    if constexpr (E == 4) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
                     "r"(r[2]), "r"(r[3])
                     : "memory");
    } else if constexpr (E == 8) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                     "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                     : "memory");
    } else {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16};" ::"r"(taddr),
            "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
            "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
            : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

template <int E>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float (&v)[E])
{
    static_assert(E == 4 || E == 8 || E == 16, "4, 8 or 16 columns");
    if constexpr (E == 16) {
        tmem_load16(taddr, v);
    } else {
        uint32_t r[E];
        if constexpr (E == 4) {
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                         : "r"(taddr));
        } else {
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(taddr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = __uint_as_float(r[i]);
    }
}

// The B operand of K-step j starts at byte vpos(j): 32 rows of 16 FP16 columns in four
// groups of 8 rows (256 bytes apart), rows 0-15 the walkers' V1 and rows 16-31 their
// V2 (V2 of walker n is row 16 + n, 512 bytes after its V1), 1 KB per K-step; one
// extra 16 bytes after every K-step puts the rows that the lanes of a quarter-warp
// write (a lane's E columns lie in K-step lane E / 16) into distinct bank groups.
__host__ __device__ constexpr uint32_t vpos(int j) { return 1040u * j; }

// Layout of the tensor-core state in dynamic shared memory (bytes from a 1024-aligned base).
struct Plan {
    int mt, ks;              // 128-row M-tiles, 16-column K-steps of d_pad
    int units;               // halves (P_hi or P_lo of one K-step, mt x 4 KB) per stage
    int npos;                // stages consumed by one contraction (2 ks / units)
    uint32_t vbytes;         // the B operands (V1 and V2 of every K-step)
    uint32_t v_off, stage_off, bar_off, total;
};

__host__ __device__ inline Plan plan(int d_pad)
{
    Plan p;
    p.mt = d_pad / 128;
    p.ks = d_pad / 16;
    p.units = static_cast<int>(STAGE_BYTES / (4096u * p.mt));
    p.npos = 2 * p.ks / p.units;
    p.vbytes = (vpos(p.ks) + 127u) & ~127u;
    p.v_off = 0;
    p.stage_off = p.v_off + p.vbytes;
    p.bar_off = p.stage_off + STAGES * STAGE_BYTES;         // full[S], empty[S], done, tmem base
    p.total = p.bar_off + (2 * STAGES + 1) * 8 + 16;
    return p;
}

// Floats of the pre-laid-out P of a run: ks K-steps x (P1, P2) x mt tiles x 4 KB of FP16.
__host__ __device__ inline long ptc_floats(int d_pad) { return 1l * d_pad * d_pad; }

// Per-CTA state (shared-memory pointers, tensor-memory base), kept in shared memory:
// thread 0 writes it, every thread reads it.
struct State {
    float *vb;            // B operands (Y^T aliases them after the MMAs)
    char *stages;
    uint64_t *full, *empty, *done;
    uint32_t *tmem_slot;
    uint32_t tmem;        // tensor-memory base address (lane 0, first column)
    uint32_t ncols;       // allocated columns: accumulators P1V1, P1V2, P2V1 of 16 columns per M-tile,
                          // then 64 columns where the walkers keep a step's momentum noise
    uint32_t noise_col;   // first noise column (warp n: lanes 32 (n % 4) .., columns + 16 (n / 4))
    const float *ptc;     // pre-laid-out P of the run (global)
    int mt, ks, units, npos;
    int *fail;            // shared failure flag
};

// Accumulator column of product k (0: P1 V1, 1: P1 V2, 2: P2 V1) of M-tile m: the N = 32
// accumulator of P1 [V1 | V2] of tile m at 32 m, that of P2 V1 at 32 mt + 16 m.
__device__ __forceinline__ uint32_t acc_col(const State &T, int k, int m)
{
    return static_cast<uint32_t>(k < 2 ? 2 * WALKERS * m + k * WALKERS : 2 * WALKERS * T.mt + WALKERS * m);
}

// The noise columns in tensor memory of the walker of warp n (lanes 32 (n % 4) .. + 31,
// which warps n, n +- 4, n +- 8, ... can address).
__device__ __forceinline__ uint32_t noise_addr(const State &T, int n)
{
    return T.tmem + (static_cast<uint32_t>(32 * (n & 3)) << 16) + T.noise_col + 16u * static_cast<uint32_t>(n >> 2);
}

// Each thread's view of the pipeline (32-bit counters, advanced incrementally): the
// stage of the next contraction's first position and, for the thread that waits on
// them, the parity of the next completion of the full barriers (MMA lane), of its
// stage's empty barrier (producer lanes) and of `done` (every thread).
struct Pipe {
    int s0 = 0;
    uint32_t full_par = 0, empty_par = 0, phase = 0;
};

__device__ __forceinline__ bool failed(const State &T) { return *reinterpret_cast<volatile int *>(T.fail) != 0; }

// Halves idx * units .. of the contraction into stage s.
__device__ __forceinline__ void fill(const State &T, int s, int idx)
{
    mbar_expect_tx(T.full + s, STAGE_BYTES);
    bulk_copy(T.stages + (size_t)s * STAGE_BYTES, T.ptc + (size_t)idx * (STAGE_BYTES / 4), STAGE_BYTES, T.full + s);
}

// CTA set-up: barriers, tensor memory, the first STAGES stages of P.  Every thread
// calls it; `T` is in shared memory; `base` is 1024-byte aligned dynamic shared memory
// of plan(d_pad).total bytes.
__device__ inline void setup(State &T, char *base, const float *ptc, int d_pad, int *fail_flag)
{
    if (threadIdx.x == 0) {
        const Plan pl = plan(d_pad);
        T.vb = reinterpret_cast<float *>(base + pl.v_off);
        T.stages = base + pl.stage_off;
        T.full = reinterpret_cast<uint64_t *>(base + pl.bar_off);
        T.empty = T.full + STAGES;
        T.done = T.empty + STAGES;
        T.tmem_slot = reinterpret_cast<uint32_t *>(T.done + 1);
        T.ptc = ptc;
        T.mt = pl.mt;
        T.ks = pl.ks;
        T.units = pl.units;
        T.npos = pl.npos;
        T.fail = fail_flag;
        T.noise_col = static_cast<uint32_t>(3 * pl.mt * WALKERS);
        uint32_t nc = 32;
        while (nc < T.noise_col + 4 * 16) nc <<= 1;  // a power of two
        T.ncols = nc;
        *fail_flag = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(T.full + s, 1);
            mbar_init(T.empty + s, 1);
        }
        mbar_init(T.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(T.tmem_slot)),
                     "r"(T.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (threadIdx.x == 0) {
        T.tmem = *T.tmem_slot;
        for (int s = 0; s < STAGES; ++s) fill(T, s, s % T.npos);
    }
    __syncthreads();
}

// CTA wind-down: the MMAs issued so far complete, the stages prefetched for a next
// contraction land, then the tensor memory is freed.  Every thread calls it.
__device__ inline void teardown(State &T, const Pipe &pp)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        mma_commit(T.done);
        if (!mbar_wait(T.done, pp.phase)) *T.fail = 1;
        int s = pp.s0;
        uint32_t par = pp.full_par;
        for (int i = 0; i < STAGES; ++i) {
            if (!mbar_wait(T.full + s, par)) *T.fail = 1;
            if (++s == STAGES) {
                s = 0;
                par ^= 1u;
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(T.tmem), "r"(T.ncols) : "memory");
}

// Lane 0 of warp 0: the MMAs of one contraction (its npos stages, the first in stage
// pp.s0) for d_pad = 128 MT.  The tile count is a compile-time constant so that the
// MMAs of a stage form one straight sequence (one lane issues them back to back;
// loop control between them slows the issue several-fold).  Within a half the
// products are issued M-tile after M-tile, each into its own accumulator;
// descriptors are built by adding shared-memory offsets (in 16-byte units) to the
// descriptor of address 0.
template <int MT>
__device__ inline void issue_mmas(const State &T, Pipe &pp)
{
    constexpr int UNITS = static_cast<int>(STAGE_BYTES / (4096u * MT));  // halves per stage
    constexpr int NPOS = 2 * (8 * MT) / UNITS;                             // stages per contraction
    constexpr uint32_t ACC_2 = 2 * MT * WALKERS;  // P2 V1 accumulators (after the N = 32 ones)
    const uint32_t idesc32 = instr_desc_f16(128, 2 * WALKERS), idesc16 = instr_desc_f16(128, WALKERS);
    const uint32_t tmem = T.tmem;
    uint64_t *const full = T.full, *const empty = T.empty;
    const uint64_t d0 = smem_desc(0, 128, 256);
    const uint32_t vb = smem_addr(T.vb) >> 4, st0 = smem_addr(T.stages) >> 4;
    int s = pp.s0;
    uint32_t par = pp.full_par;
#pragma unroll 1
    for (int i = 0; i < NPOS; ++i) {
        if (failed(T) || !mbar_poll(full + s, par)) {
            *T.fail = 1;
            return;
        }
        fence_after_sync();
        const uint32_t sa = st0 + static_cast<uint32_t>(s) * (STAGE_BYTES >> 4);
#pragma unroll
        for (int u = 0; u < UNITS; ++u) {
            const int q = i * UNITS + u;  // half: K-step q / 2, P2 if q odd
            const int j = q >> 1;
            const uint32_t vj = vpos(j) >> 4;
            const uint32_t acc = j > 0 ? 1u : 0u;
            const uint64_t b = d0 + vb + vj;  // rows 0-15 (V1), or 0-31 (V1 and V2) with N = 32
            const uint64_t a0 = d0 + sa + static_cast<uint32_t>(u * MT) * 256u;
            if ((q & 1) == 0) {
#pragma unroll
                for (int m = 0; m < MT; ++m) mma_f16(tmem + 2 * WALKERS * m, a0 + 256u * m, b, idesc32, acc);
            } else {
#pragma unroll
                for (int m = 0; m < MT; ++m) mma_f16(tmem + ACC_2 + m * WALKERS, a0 + 256u * m, b, idesc16, acc);
            }
        }
        mma_commit(empty + s);
        if (++s == STAGES) {
            s = 0;
            par ^= 1u;
        }
    }
    pp.full_par = par;
    mma_commit(T.done);
}

// Lane 0 of warp 1 + w: the refills of stage w during one contraction (positions
// STAGES .. npos + STAGES - 1 of the contraction, counted from its first, that fall
// in stage w; those past npos prefetch the next contraction), each once the MMAs
// that read the stage's previous content are done.
__device__ inline void refill_stage(const State &T, Pipe &pp, int w)
{
    int idx = STAGES + (w - pp.s0 + STAGES) % STAGES;
    for (; idx < T.npos + STAGES; idx += STAGES) {
        if (failed(T) || !mbar_poll(T.empty + w, pp.empty_par)) {
            *T.fail = 1;
            return;
        }
        pp.empty_par ^= 1u;
        fill(T, w, idx % T.npos);  // npos may be below STAGES (d_pad 128): one block ahead or more
    }
}

// y = P v for the 16 walkers of the CTA (lane l of warp n holds components l E ..
// l E + E - 1 of walker n).  sv is the power of two s_v that scales v before the split
// and tinv = 1 / (s_p s_v).  Every thread of the CTA calls it (barriers inside).
// Returns false if a wait gave up (y is then undefined).
// `idle()` runs in the warps that neither issue MMAs nor refill stages, while the
// contraction streams (work that the step needs later and that does not depend on y).
template <int E, class Idle>
__device__ inline bool contract(const State &T, Pipe &pp, const float (&v)[E], int d_pad, float sv, float tinv,
                                float (&y)[E], const Idle &idle)
{
    static_assert(E % 4 == 0, "quads of columns");
    static_assert(STAGES + 1 <= WALKERS, "a producer warp per stage besides the issuing warp");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // B operand: columns c .. c + 3 of walker n (8 bytes of FP16) lie in row n % 8 of
    // core matrix (c % 16) / 8 of walker group n / 8 in K-step c / 16, at byte 2 (c % 8)
    char *vh = reinterpret_cast<char *>(T.vb), *vl = vh + 512;  // V2 of walker n is row 16 + n
    const uint32_t row_off = static_cast<uint32_t>((warp >> 3) * 256 + (warp & 7) * 16);
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
        const int c = lane * E + 4 * q;
        const uint32_t off = vpos(c >> 4) + row_off + static_cast<uint32_t>(((c >> 3) & 1) * 128 + (c & 7) * 2);
        float h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float t = v[4 * q + i] * sv;
            h[i] = __half2float(__float2half_rn(t));
            l[i] = (t - h[i]) * 2048.f;  // exact: t - h[i] is representable
        }
        *reinterpret_cast<uint2 *>(vh + off) = make_uint2(pack_half2(h[0], h[1]), pack_half2(h[2], h[3]));
        *reinterpret_cast<uint2 *>(vl + off) = make_uint2(pack_half2(l[0], l[1]), pack_half2(l[2], l[3]));
    }
    fence_async_smem();
    __syncthreads();
    if (warp <= STAGES) {
        // the working lane's warp-mates wait at the warp barrier, not in a blocking
        // mbarrier test that would hold the working lane's warp as well
        if (lane == 0) {
            if (warp == 0) {
                fence_after_sync();
                issue_mmas<E / 4>(T, pp);  // d_pad = 32 E = 128 (E / 4) rows
            } else {
                refill_stage(T, pp, warp - 1);
            }
        }
        __syncwarp();
    } else {
        idle();
    }
    pp.s0 = (pp.s0 + T.npos) % STAGES;
    // every thread: the accumulators are complete
    const bool ok = !failed(T) && mbar_wait(T.done, pp.phase);
    pp.phase ^= 1u;
    fence_after_sync();
    // Y^T[walker][d_pad] over the B operands (free once the MMAs are done; vbytes >=
    // 65 d_pad bytes), each walker's row in the lane-row layout so that the walker reads
    // it back in quads
    float *ybuf = T.vb;
    if (ok && warp < 4 * T.mt) {
        const int m = warp >> 2, q = warp & 3;
        const uint32_t lanes = static_cast<uint32_t>(32 * q) << 16;
        float a11[16], a12[16], a21[16];
        tmem_load16(T.tmem + lanes + acc_col(T, 0, m), a11);
        tmem_load16(T.tmem + lanes + acc_col(T, 1, m), a12);
        tmem_load16(T.tmem + lanes + acc_col(T, 2, m), a21);
        const int row = swz_col<E>(m * 128 + 32 * q + lane);
#pragma unroll
        for (int n = 0; n < WALKERS; ++n) ybuf[n * d_pad + row] = fmaf(a12[n] + a21[n], 0x1p-11f, a11[n]) * tinv;
    }
    fence_before_sync();
    __syncthreads();
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
        const float4 t = lane_quad<E>(ybuf + warp * d_pad, lane, q);
        y[4 * q] = t.x;
        y[4 * q + 1] = t.y;
        y[4 * q + 2] = t.z;
        y[4 * q + 3] = t.w;
    }
    __syncthreads();  // ybuf is the next contraction's B operand
    return ok && !failed(T);
}

}  // namespace tc
}  // namespace ggns
