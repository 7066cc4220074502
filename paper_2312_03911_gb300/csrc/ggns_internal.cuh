// ggns_internal.cuh -- device data layout and helpers shared by the CUDA
// translation units of libggns (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ggns.h"

namespace ggns {

constexpr int CMAX = 64;        // cluster slots per run
constexpr int KNN_K = 16;       // neighbour ranks precomputed per point for Algorithm 4 (later ranks: exact scan)
constexpr int NLIVE_MAX = 16384;
constexpr int KMAX_COMP = 64;   // mixture components
constexpr int DMAX = 512;
constexpr int WINT = 16;        // ints of walker state per walker (three-phase HSS)

// Philox counter purposes (the fourth counter word is (iteration << 4) | purpose).
enum Purpose : uint32_t {
    P_INIT = 0, P_MOM = 1, P_NOISE = 2, P_RES = 3, P_CLUSTER = 4, P_START = 5, P_PRUNE = 6
};

// Walker tile: G lanes per walker, E components per lane (d <= G*E).
struct Tile {
    int g, e;
};

// Step records of the single-pass HSS (one row per walker-step).
struct RecView {
    uint2 *meta;
    float *ll;
    float *x;
    int rec_len;  // records per walker
    int xs;       // floats per x record (the largest d_pad of the batch)
    // momentum noise drawn ahead by k_noise: normals z[(walker row * nT + step - 1) * xs + c]
    // and the reservoir words sp[walker row * nT + step - 1]; nT = 0: drawn in the walk
    float *nz;
    uint32_t *nsp;
    int nT;
    int pad_;
};

// Steps of noise drawn ahead for an iteration: all nT for the first iteration,
// then 1.1 x the previous t_stop + 4 (at most nT); later steps draw inline.  The
// draw competes with the k-NN for the SMs, so a tight estimate pays (t_stop moves
// little between iterations).
__host__ __device__ inline int noise_steps(int nT, int t_stop_last)
{
    if (t_stop_last <= 0) return nT;
    const int n = t_stop_last + t_stop_last / 10 + 4;
    return n < nT ? n : nT;
}

// Constant description of one run (device copy, read by every kernel).
struct RunDesc {
    int d, d_pad, n_live, k, kind, n_comp;
    int n_steps, min_steps, min_ref, max_ref, prune_after, termination, clustering, noise_mode;
    int noise_inside, pick_all, territory, keep_last;  // readings of Algorithm 5 (ns_config)
    int box_fold, fold_counts;                         // exact reflection off the prior box; its
                                                       // reflections in the step-size control
    int midpoint;                                      // the time-reversible step (half move, reflection
                                                       // at the half step, half move)
    float delta_p, keep, rosen_scale, lik_const;
    float torus_a, torus_b, torus_c;  // TORUS: sine and cosine frequencies, offset
    float tc_sv, tc_inv;              // tensor-core contraction: scale s_v of v, 1 / (s_p s_v)
    double log_tol, out_lo, out_hi, dt_init;
    uint32_t key0, key1;
    long max_iters;
    // offsets (elements) into the context arenas
    long x_off;      // live x   [n_live][d_pad]         float arena
    long pt_off;     // per-point arrays [n_live]          (logl float / label int / order int)
    long w_off;      // per-walker arrays [k]              (start slot, new label, walker ints)
    long ws_off;     // walker float state [k][3 d_pad]    float arena
    long par_off;    // likelihood parameter block         float arena
    long dead_off;   // first dead row of this run in its arrays (0: one allocation per run)
    long dead_cap;   // rows available in the dead arrays
    float *dead_x;   // [dead_cap][d_pad]  (reallocated by the host as the run grows)
    float *dead_logl;
    double *dead_logw;
    int *dead_label;
    long nbr_off;    // k-NN ranks [n_live][KNN_K]         int arena
    int tile;        // walker tile id
    int pad_;
};

// Layout of the float parameter block of one run (offsets from par_off):
//   lo[d_pad], hi[d_pad], means[n_comp][d_pad], comp_a[n_comp], comp_b[n_comp],
//   precision[d][d_pad] (dense kinds), pmu[n_comp][d_pad] (dense mixture: P mu_k).
// comp_a/comp_b: ISO kinds: a = 1/sigma^2, b = log w_k - d/2 log(2 pi sigma^2);
//                dense kinds: a unused, b = log w_k (mixture), 0 (single Gaussian).
struct ParLayout {
    long lo, hi, means, comp_a, comp_b, prec, pmu, ptc, total;
};
// Dense kinds whose d_pad is 128, 256 or 512 also carry P scaled by a power of two s_p and
// pre-split into FP16 pairs s_p P = P1 + 2^-11 P2, laid out for the tensor cores
// (ggns_tc.cuh): d_pad/16 K-steps x (P1, P2) x d_pad/128 tiles of 128 rows x 16 columns in
// core-matrix order (d_pad^2 floats' worth of FP16, global memory only).
__host__ __device__ inline bool tc_layout(int kind, int d_pad)
{
    return (kind == NS_LIK_DENSE_GAUSS || kind == NS_LIK_DENSE_MIX) && d_pad % 128 == 0 && d_pad <= 512;
}
// Component slots of the parameter block: an isotropic mixture of up to 8
// components is padded to 4 or 8 slots (a = 0, b = -inf, mean 0: weight exactly
// 0), so its likelihood runs over a compile-time count.
// Kinds without component means (ROSENBROCK, TORUS): one parameter-free component.
__host__ __device__ inline bool kind_has_means(int kind)
{
    return kind != NS_LIK_ROSENBROCK && kind != NS_LIK_TORUS;
}

__host__ __device__ inline int comp_slots(int n_comp, int kind)
{
    if (kind == NS_LIK_MIX_ISO && n_comp <= 8) return n_comp <= 4 ? 4 : 8;
    return n_comp;
}

__host__ __device__ inline ParLayout par_layout(int d, int d_pad, int n_comp, int kind)
{
    ParLayout L;
    long o = 0;
    const int ns = comp_slots(n_comp, kind);
    L.lo = o; o += d_pad;
    L.hi = o; o += d_pad;
    L.means = o; o += (long)ns * d_pad;
    L.comp_a = o; o += ns;
    L.comp_b = o; o += ns;
    o = (o + 3) & ~3L;
    L.prec = o;
    if (kind == NS_LIK_DENSE_GAUSS || kind == NS_LIK_DENSE_MIX) o += (long)d * d_pad;
    L.pmu = o;
    if (kind == NS_LIK_DENSE_MIX) o += (long)n_comp * d_pad;
    o = (o + 3) & ~3L;  // 16-byte aligned: the tensor-core layout is read by bulk copies
    L.ptc = o;
    if (tc_layout(kind, d_pad)) o += 1l * d_pad * d_pad;
    L.total = (o + 3) & ~3L;
    return L;
}

// Mutable per-run state.
struct RunState {
    int iter, done, status, terminated;
    int n_clusters, max_clusters, t_save, t_stop;
    double dt, log_xl, log_xl_max, lstar;
    long n_dead, n_like, n_steps_total, n_in, n_out;
    unsigned int wcount[3]; // walker refill counters of the three HSS phases
    int final_done;
    int n_fallback;
    double logz, logz2;
    long dead_base;        // first dead row of the current iteration's kills
    int ev_pending;        // the iteration's statistics update has not run yet
    int remain_min;        // single-pass HSS: walkers yet to reach min_ref
    int remain_max;        // single-pass HSS: walkers yet to meet their stop rule
    int rec_overflow;      // single-pass HSS ran out of record length: redo in three phases
    unsigned int wcount1;  // single-pass HSS walker refill counter
    int t_save1, t_stop1;  // single-pass HSS window
    int t_stop_last;       // t_stop of the previous iteration (sizes the noise drawn ahead)
    int term_pending;      // the iteration's tail ran; its termination test waits for the statistics
    float lmax_live;       // L_max over the live points after the iteration (classic termination)
    int n_rec_overflow;    // iterations redone in three phases
    int kill_cnt[CMAX];    // kills per cluster in the current iteration
    int spawn_cnt[CMAX];   // new points per cluster in the current iteration
    long n_fold;           // inside steps on which the box reflected the walker (box_fold)
};

// Checked builds (compiled with -DGGNS_CHECKED, the stand-in for a memory checker):
// indexes into the dead-point arena, the step records and the live slots are checked
// before the access; a failed check skips the access and leaves NS_ERR_BOUNDS in the
// run's status, which the host reports like any other status.  In the default build
// the check is the constant true.
#ifdef GGNS_CHECKED
__device__ __forceinline__ bool gg_in(long i, long n, RunState *S)
{
    if (i >= 0 && i < n) return true;
    atomicCAS(&S->status, 0, static_cast<int>(NS_ERR_BOUNDS));
    return false;
}
#else
__device__ __forceinline__ bool gg_in(long, long, RunState *) { return true; }
#endif

// FP64 cluster statistics of one run (Appendix H), log space.
struct Stats {
    double logZp[CMAX], logZp2[CMAX], logZXp[CMAX], logZpXp[CMAX], logXp[CMAX], logXp2[CMAX];
    double logXX[CMAX * CMAX];
    int n[CMAX];
    int alive[CMAX];
};

// Device view of a context.
struct DevCtx {
    int n_runs;
    const RunDesc *desc;
    RunState *state;
    Stats *stats;
    float *fa;        // float arena: live x, walker float state, parameters
    float *logl;      // [sum n_live]
    int *label;       // [sum n_live]
    int *order;       // [sum n_live]  ascending (logL, slot) order of the last selection
    int *start_slot;  // [sum k]
    int *new_label;   // [sum k]
    int *wint;        // [sum k][WINT]  walker integer state
    float *wres_logl; // [sum k]
    int *nbr;         // [sum n_live][KNN_K]
};

// ------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
    }
    return c;
}

__device__ __forceinline__ U4 rng_block(const RunDesc &D, uint32_t iter, uint32_t purpose, uint32_t slot,
                                        uint32_t step, uint32_t block)
{
    U4 c{block, step, slot, (iter << 4) | purpose};
    return philox4x32_10(c, D.key0, D.key1);
}

// (0,1) uniform from the top 23 bits plus one half: exact in FP32.
__device__ __forceinline__ float u01(uint32_t r)
{
    return (static_cast<float>(r >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

// FP64 uniform from 52 bits plus one half.
__device__ __forceinline__ double u01_52(uint32_t r0, uint32_t r1)
{
    const uint64_t m = (static_cast<uint64_t>(r0) << 20) | static_cast<uint64_t>(r1 >> 12);
    return (static_cast<double>(m) + 0.5) * (1.0 / 4503599627370496.0);
}

// Box-Muller pair from two words.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &z0, float &z1)
{
    const float rad = sqrtf(-2.0f * logf(u01(a)));
    float s, c;
    sincospif(2.0f * u01(b), &s, &c);
    z0 = rad * c;
    z1 = rad * s;
}

// 32 bits from the low 9 bits of the four words of a block: the bits the
// uniforms below do not use (they take the top 23 bits of each word).
__device__ __forceinline__ uint32_t spare_bits(const U4 &w)
{
    return (w.x & 511u) | ((w.y & 511u) << 9) | ((w.z & 511u) << 18) | ((w.w & 31u) << 27);
}

// The E normals of components c0 .. c0+E-1 (c0 a multiple of E; E in {1,2,4,8,16}).
// *spare (may be null) receives spare_bits of the lane's first block.
template <int E>
__device__ __forceinline__ void lane_normals(const RunDesc &D, uint32_t iter, uint32_t purpose, uint32_t slot,
                                             uint32_t step, int c0, float (&z)[E], uint32_t *spare = nullptr)
{
    if constexpr (E >= 4) {
#pragma unroll
        for (int b = 0; b < E / 4; ++b) {
            const U4 w = rng_block(D, iter, purpose, slot, step, static_cast<uint32_t>((c0 >> 2) + b));
            if (b == 0 && spare) *spare = spare_bits(w);
            box_muller(w.x, w.y, z[4 * b + 0], z[4 * b + 1]);
            box_muller(w.z, w.w, z[4 * b + 2], z[4 * b + 3]);
        }
    } else {
        const U4 w = rng_block(D, iter, purpose, slot, step, static_cast<uint32_t>(c0 >> 2));
        if (spare) *spare = spare_bits(w);
        const int off = c0 & 3;
        float a0, a1;
        if (off < 2) box_muller(w.x, w.y, a0, a1);
        else box_muller(w.z, w.w, a0, a1);
        if constexpr (E == 2) {
            z[0] = a0;
            z[1] = a1;
        } else {
            z[0] = (off & 1) ? a1 : a0;
        }
    }
}

// ------------------------------------------------------------------------
// Group reductions (G lanes of one warp, all 32 lanes execute them)
// ------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ float gsum(float v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ int gsum_i(int v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ float gmax(float v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ------------------------------------------------------------------------
// Lane rows in shared memory.  In the one-walker-per-warp kernels lane l holds the
// E = d_pad / 32 consecutive components l E .. l E + E - 1, so a warp reading "its"
// element e of a per-component vector hits addresses E floats apart: for E = 16
// sixteen lanes share each bank.  A vector kept in shared memory for such a warp is
// stored with the 16-byte quads of each lane row permuted: quad q of lane l sits at
// quad q ^ qswz(l) of the row.  A quarter-warp (the eight lanes one 16-byte access
// serves per pass) then reads quad q through eight distinct bank groups.
// ------------------------------------------------------------------------
template <int E>
__host__ __device__ constexpr int qswz(int l)
{
    constexpr int m = E / 4;          // quads per lane row
    constexpr int p2 = m & -m;        // largest power of two dividing m
    constexpr int p = p2 > 8 ? 8 : p2;
    if constexpr (E % 4 != 0 || p == 1) {
        return 0;                     // odd quad counts reach eight bank groups unpermuted
    } else if constexpr (p == 8) {
        return l & 7;
    } else {
        return ((l * p) >> 3) & (p - 1);
    }
}

// Stored position of component c of a lane-row-permuted vector.
template <int E>
__host__ __device__ constexpr int swz_col(int c)
{
    if constexpr (E % 4 != 0) {
        return c;
    } else {
        const int l = c / E, w = c - l * E;
        return l * E + (((w >> 2) ^ qswz<E>(l)) << 2) + (w & 3);
    }
}

// Quad q (components lane E + 4 q .. + 3) of a lane-row-permuted vector `row`.
template <int E>
__device__ __forceinline__ float4 lane_quad(const float *row, int lane, int q)
{
    return reinterpret_cast<const float4 *>(row + lane * E)[q ^ qswz<E>(lane)];
}

// Permute `nrows` vectors of `len` floats (consecutive, 16-byte aligned, len a
// multiple of 32 E) in shared memory into the lane-row layout.  Call by the whole
// CTA; the caller synchronises afterwards.
template <int E>
__device__ inline void swizzle_rows(float *base, int nrows, int len)
{
    if constexpr (E % 4 == 0 && qswz<E>(1) + qswz<E>(2) + qswz<E>(4) != 0) {
        const int qpr = len / 4;      // quads per vector
        float4 *b4 = reinterpret_cast<float4 *>(base);
        for (int i = threadIdx.x; i < nrows * qpr; i += blockDim.x) {
            const int qi = i % qpr;
            const int l = qi / (E / 4), q = qi - l * (E / 4);
            const int q2 = q ^ qswz<E>(l % 32);
            if (q2 > q) {
                const int j = i - q + q2;
                const float4 t = b4[i];
                b4[i] = b4[j];
                b4[j] = t;
            }
        }
    }
}

// Order-preserving 32-bit key of a float; NaN maps to 0 (sorts first).
__device__ __forceinline__ uint32_t float_key(float f)
{
    if (f != f) return 0u;
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ double log_add(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    const double m = a > b ? a : b;
    return m + log1p(exp(-fabs(a - b)));
}

}  // namespace ggns
