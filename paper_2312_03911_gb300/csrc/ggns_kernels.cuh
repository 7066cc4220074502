// ggns_kernels.cuh -- walker-layout kernels templated on the likelihood kind and
// the walker tile (G lanes per walker, E components per lane).  Each kind is
// instantiated in its own translation unit (ggns_k_<kind>.cu).
#pragma once

#include "ggns_internal.cuh"
#include "ggns_tc.cuh"

namespace ggns {

constexpr int HSS_THREADS = 128;

// Shared-memory view of a run's likelihood parameters.
struct ParView {
    const float *lo, *hi, *means, *a, *b, *prec, *pmu;
    const float *ptc;  // P for the tensor cores (global memory; dense kinds with d_pad 128, 256, 512)
};

// Periodic prior (TORUS): wrap each real component of x into [lo, hi) after a move,
// so the walker never leaves the prior (padded components stay at 0).
template <int KIND, int E>
__device__ __forceinline__ void wrap_periodic(const RunDesc &D, const ParView &P, float (&x)[E], int c0)
{
    if constexpr (KIND == NS_LIK_TORUS) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int c = c0 + e;
            if (c < D.d) {
                const float lo = P.lo[c], w = P.hi[c] - lo;
                float u = x[e] - lo;
                u -= w * floorf(u / w);
                if (u >= w) u -= w;  // rounding of the quotient
                if (u < 0.f) u = 0.f;
                x[e] = lo + u;
            }
        }
    }
}

// Prior box with box_fold: a component that left [lo, hi] is reflected back exactly
// (the path unfolded on a line of period 2w folds into the box; an odd number of
// crossings flips that momentum component), so the walker never leaves the prior
// and the box takes no outside step.  Padded components (lo = hi = x = 0) never fold.
// SWZ: lo and hi are in the lane-row layout (one-walker-per-warp kernels).  Returns
// whether one of this lane's components folded.
template <int KIND, int E, bool SWZ = false>
__device__ __forceinline__ bool fold_box(const RunDesc &D, const ParView &P, float (&x)[E], float (&p)[E], int c0)
{
    bool folded = false;
    if constexpr (KIND != NS_LIK_TORUS) {
        if (!D.box_fold) return false;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int c = SWZ ? swz_col<E>(c0 + e) : c0 + e;
            const float lo = P.lo[c], hi = P.hi[c];
            if (!(x[e] < lo || x[e] > hi)) continue;
            folded = true;
            const float w = hi - lo, w2 = 2.f * w;
            float u = x[e] - lo;
            u -= w2 * floorf(u / w2);
            if (u >= w2) u -= w2;  // rounding of the quotient
            if (u < 0.f) u = 0.f;
            if (u > w) {
                x[e] = lo + (w2 - u);
                p[e] = -p[e];
            } else {
                x[e] = lo + u;
            }
        }
    }
    return folded;
}

// Copy the parameter block of run D into shared memory (the precision matrix
// only when `prec_in_smem`); returns the view.  Call by the whole CTA.
__device__ inline ParView load_params(const DevCtx &C, const RunDesc &D, float *sm, bool prec_in_smem)
{
    const ParLayout L = par_layout(D.d, D.d_pad, D.n_comp, D.kind);
    const float *gp = C.fa + D.par_off;
    const long n_small = L.prec;  // lo, hi, means, a, b
    for (long i = threadIdx.x; i < n_small; i += blockDim.x) sm[i] = gp[i];
    long o = n_small;
    ParView v;
    v.lo = sm + L.lo;
    v.hi = sm + L.hi;
    v.means = sm + L.means;
    v.a = sm + L.comp_a;
    v.b = sm + L.comp_b;
    const long n_prec = L.pmu - L.prec;
    if (n_prec > 0 && prec_in_smem) {
        for (long i = threadIdx.x; i < n_prec; i += blockDim.x) sm[o + i] = gp[L.prec + i];
        v.prec = sm + o;
        o += n_prec;
    } else {
        v.prec = gp + L.prec;
    }
    const long n_pmu = L.ptc - L.pmu;
    if (n_pmu > 0) {
        for (long i = threadIdx.x; i < n_pmu; i += blockDim.x) sm[o + i] = gp[L.pmu + i];
        v.pmu = sm + o;
        o += n_pmu;
    } else {
        v.pmu = nullptr;
    }
    v.ptc = (L.total > L.ptc) ? gp + L.ptc : nullptr;
    return v;
}

// Shared memory (floats) needed by load_params.
__host__ __device__ inline long param_smem_floats(const RunDesc &D, bool prec_in_smem)
{
    const ParLayout L = par_layout(D.d, D.d_pad, D.n_comp, D.kind);
    long n = L.prec + (L.ptc - L.pmu);
    if (prec_in_smem) n += L.pmu - L.prec;
    return n;
}

// ------------------------------------------------------------------------
// Fused log-likelihood and score (Section 2.3: only the direction of the
// score enters the reflection; the value decides inside/outside).
// x, g: the E components c0 .. c0+E-1 of one walker held by this lane.
// rbuf: per-walker shared scratch of d_pad floats (dense kinds only).
// resp: optional responsibilities per component (for d/d mu), or nullptr.
// ------------------------------------------------------------------------
// Isotropic mixture over KS padded component slots (KS compile-time: straight-line
// code; padded slots have weight exactly 0).  Distances for every slot, one
// max, one normalisation; exp, log and the reciprocal use the SFU forms (a few
// ulp; the log-likelihood is used to FP32 accuracy anyway).
template <int KS, int G, int E>
__device__ __forceinline__ float lik_mix_slots(const ParView &P, int dp, const float (&x)[E], float (&g)[E], int c0,
                                               int K, float *dmu_w)
{
    float q[KS], tk[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        q[k] = 0.f;
        const float *mu = P.means + (long)k * dp + c0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float r = x[e] - mu[e];
            q[k] = fmaf(r, r, q[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < KS; ++k) q[k] = gsum<G>(q[k]);
    float m = -INFINITY;
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        tk[k] = P.b[k] - 0.5f * P.a[k] * q[k];
        m = fmaxf(m, tk[k]);
    }
    float s = 0.f, acc[E];
#pragma unroll
    for (int e = 0; e < E; ++e) acc[e] = 0.f;
#pragma unroll
    for (int k = 0; k < KS; ++k) {
        const float wk = __expf(tk[k] - m);
        s += wk;
        if (dmu_w && k < K) dmu_w[k] = wk;
        const float *mu = P.means + (long)k * dp + c0;
        const float c = -wk * P.a[k];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = fmaf(c, x[e] - mu[e], acc[e]);
    }
    const float inv = __fdividef(1.f, s);
#pragma unroll
    for (int e = 0; e < E; ++e) g[e] = acc[e] * inv;
    if (dmu_w)
        for (int k = 0; k < K; ++k) dmu_w[k] *= inv;
    return m + __logf(s);
}

// Dense kinds after y = P v (v = x - mu, or x for the mixture): the quadratic
// forms, the log-sum-exp over the components and the score.  SWZ: one walker per
// warp (G = 32) with means and P mu in the lane-row layout, read as quads.
template <int KIND, int G, int E, bool SWZ = false>
__device__ __forceinline__ float dense_finish(const RunDesc &D, const ParView &P, const float (&x)[E],
                                              const float (&y)[E], float (&g)[E], int c0, float *dmu_w)
{
    static_assert(!SWZ || (G == 32 && E % 4 == 0), "lane rows of whole quads");
    const int dp = D.d_pad;
    const bool mix = (KIND == NS_LIK_DENSE_MIX);
    const int K = mix ? D.n_comp : 1;
    const int lane = threadIdx.x & 31;
    if (!mix) {
        float q = 0.f;
        if constexpr (SWZ) {
#pragma unroll
            for (int h = 0; h < E / 4; ++h) {
                const float4 mu = lane_quad<E>(P.means, lane, h);
                q = fmaf(x[4 * h] - mu.x, y[4 * h], q);
                q = fmaf(x[4 * h + 1] - mu.y, y[4 * h + 1], q);
                q = fmaf(x[4 * h + 2] - mu.z, y[4 * h + 2], q);
                q = fmaf(x[4 * h + 3] - mu.w, y[4 * h + 3], q);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) q = fmaf(x[e] - P.means[c0 + e], y[e], q);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) g[e] = -y[e];
        q = gsum<G>(q);
        if (dmu_w) dmu_w[0] = 1.f;
        return D.lik_const - 0.5f * q;
    }
    // g accumulates the responsibility-weighted -(y - P mu_k), rescaled as the maximum moves
    float m = -INFINITY, s = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) g[e] = 0.f;
    for (int k = 0; k < K; ++k) {
        const float *mu = P.means + (long)k * dp;
        const float *pm = P.pmu + (long)k * dp;
        float q = 0.f;
        if constexpr (SWZ) {
#pragma unroll
            for (int h = 0; h < E / 4; ++h) {
                const float4 a = lane_quad<E>(mu, lane, h), b = lane_quad<E>(pm, lane, h);
                q = fmaf(x[4 * h] - a.x, y[4 * h] - b.x, q);
                q = fmaf(x[4 * h + 1] - a.y, y[4 * h + 1] - b.y, q);
                q = fmaf(x[4 * h + 2] - a.z, y[4 * h + 2] - b.z, q);
                q = fmaf(x[4 * h + 3] - a.w, y[4 * h + 3] - b.w, q);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) q = fmaf(x[e] - mu[c0 + e], y[e] - pm[c0 + e], q);
        }
        q = gsum<G>(q);
        const float tk = P.b[k] - 0.5f * q;
        if (tk > m) {
            const float sc = (m == -INFINITY) ? 0.f : expf(m - tk);
            s *= sc;
#pragma unroll
            for (int e = 0; e < E; ++e) g[e] *= sc;
            m = tk;
        }
        const float wk = expf(tk - m);
        s += wk;
        if constexpr (SWZ) {
#pragma unroll
            for (int h = 0; h < E / 4; ++h) {
                const float4 b = lane_quad<E>(pm, lane, h);
                g[4 * h] = fmaf(-wk, y[4 * h] - b.x, g[4 * h]);
                g[4 * h + 1] = fmaf(-wk, y[4 * h + 1] - b.y, g[4 * h + 1]);
                g[4 * h + 2] = fmaf(-wk, y[4 * h + 2] - b.z, g[4 * h + 2]);
                g[4 * h + 3] = fmaf(-wk, y[4 * h + 3] - b.w, g[4 * h + 3]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) g[e] = fmaf(-wk, y[e] - pm[c0 + e], g[e]);
        }
        if (dmu_w) dmu_w[k] = tk;
    }
    const float inv = 1.f / s;
#pragma unroll
    for (int e = 0; e < E; ++e) g[e] *= inv;
    if (dmu_w) {
        for (int k = 0; k < K; ++k) dmu_w[k] = expf(dmu_w[k] - m) * inv;
    }
    return D.lik_const + m + logf(s);
}

template <int KIND, int G, int E>
__device__ __forceinline__ float lik_eval(const RunDesc &D, const ParView &P, const float (&x)[E], float (&g)[E],
                                          int c0, float *rbuf, float *dmu_w)
{
    const int d = D.d;
    const int dp = D.d_pad;
    if constexpr (KIND == NS_LIK_ISO_GAUSS) {
        const float a = P.a[0];
        float q = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float r = x[e] - P.means[c0 + e];  // padded components: x = mu = 0
            q = fmaf(r, r, q);
            g[e] = -a * r;
        }
        q = gsum<G>(q);
        return P.b[0] - 0.5f * a * q;
    } else if constexpr (KIND == NS_LIK_MIX_ISO) {
        constexpr int KC = 8;
        const int K = D.n_comp;
        if (K <= 4) return lik_mix_slots<4, G, E>(P, dp, x, g, c0, K, dmu_w);
        if (K <= 8) return lik_mix_slots<8, G, E>(P, dp, x, g, c0, K, dmu_w);
        // more components: online log-sum-exp over chunks of KC
        float m = -INFINITY, s = 0.f;
        float acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        for (int k0 = 0; k0 < K; k0 += KC) {
            float q[KC];
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                q[kk] = 0.f;
                if (k0 + kk < K) {
                    const float *mu = P.means + (long)(k0 + kk) * dp + c0;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const float r = x[e] - mu[e];
                        q[kk] = fmaf(r, r, q[kk]);
                    }
                }
            }
#pragma unroll
            for (int kk = 0; kk < KC; ++kk)
                if (k0 + kk < K) q[kk] = gsum<G>(q[kk]);
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                if (k0 + kk < K) {
                    const int k = k0 + kk;
                    const float tk = P.b[k] - 0.5f * P.a[k] * q[kk];
                    if (tk > m) {
                        const float sc = (m == -INFINITY) ? 0.f : expf(m - tk);
                        s *= sc;
#pragma unroll
                        for (int e = 0; e < E; ++e) acc[e] *= sc;
                        m = tk;
                    }
                    const float wk = expf(tk - m);
                    s += wk;
                    const float *mu = P.means + (long)k * dp + c0;
                    const float ak = P.a[k];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const float r = x[e] - mu[e];
                        acc[e] = fmaf(-wk * ak, r, acc[e]);
                    }
                }
            }
        }
        const float inv = 1.f / s;
#pragma unroll
        for (int e = 0; e < E; ++e) g[e] = acc[e] * inv;
        if (dmu_w) {
            for (int k = 0; k < K; ++k) {
                const float *mu = P.means + (long)k * dp + c0;
                float qk = 0.f;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const float r = x[e] - mu[e];
                    qk = fmaf(r, r, qk);
                }
                qk = gsum<G>(qk);
                dmu_w[k] = expf(P.b[k] - 0.5f * P.a[k] * qk - m) * inv;
            }
        }
        return m + logf(s);
    } else if constexpr (KIND == NS_LIK_ROSENBROCK) {
        const float sc = D.rosen_scale;
        const float xn = __shfl_down_sync(0xffffffffu, x[0], 1);
        const float xp = __shfl_up_sync(0xffffffffu, x[E - 1], 1);
        float s = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int c = c0 + e;
            const float nxt = (e < E - 1) ? x[(e + 1) < E ? e + 1 : e] : xn;
            const float prv = (e > 0) ? x[e > 0 ? e - 1 : 0] : xp;
            float ge = 0.f;
            if (c < d - 1) {
                const float a = nxt - x[e] * x[e];
                const float b = 1.f - x[e];
                s = fmaf(100.f * a, a, fmaf(b, b, s));
                ge += -sc * (-400.f * x[e] * a - 2.f * b);
            }
            if (c >= 1 && c < d) {
                const float ap = x[e] - prv * prv;
                ge += -sc * (200.f * ap);
            }
            g[e] = ge;
        }
        s = gsum<G>(s);
        return -sc * s;
    } else if constexpr (KIND == NS_LIK_TORUS) {
        // eq. torus: S = sum of sin(alpha x) over the paper's even (1-based) coordinates, i.e.
        // the 0-based odd ones, + sum of cos(beta x) over the others + c; log L = 3 log S and
        // d log L / dx = (3 / S) dS / dx
        float s = 0.f, ds[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int c = c0 + e;
            ds[e] = 0.f;
            if (c < d) {
                float sn, cs;
                if (c & 1) {
                    sincosf(D.torus_a * x[e], &sn, &cs);
                    s += sn;
                    ds[e] = D.torus_a * cs;
                } else {
                    sincosf(D.torus_b * x[e], &sn, &cs);
                    s += cs;
                    ds[e] = -D.torus_b * sn;
                }
            }
        }
        s = gsum<G>(s) + D.torus_c;
        if (!(s > 0.f)) {
#pragma unroll
            for (int e = 0; e < E; ++e) g[e] = 0.f;
            return -INFINITY;
        }
        const float k3 = 3.f / s;
#pragma unroll
        for (int e = 0; e < E; ++e) g[e] = k3 * ds[e];
        return 3.f * logf(s);
    } else {
        // dense kinds: y = P v on CUDA cores, v staged through the walker's shared buffer
        const bool mix = (KIND == NS_LIK_DENSE_MIX);
        // stage v = x - mu (single Gaussian) or x (mixture: P x, then subtract P mu_k)
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int c = c0 + e;
            float v = 0.f;
            if (c < d) v = mix ? x[e] : x[e] - P.means[c];
            rbuf[c] = v;
        }
        __syncwarp();
        float y[E];
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] = 0.f;
        for (int j = 0; j < d; ++j) {
            const float vj = rbuf[j];
            const float *row = P.prec + (long)j * dp + c0;  // P symmetric: row j, columns c0..
#pragma unroll
            for (int e = 0; e < E; ++e) y[e] = fmaf(row[e], vj, y[e]);
        }
        __syncwarp();
        return dense_finish<KIND, G, E>(D, P, x, y, g, c0, dmu_w);
    }
}

// Dense likelihood of every walker of a CTA at once (one walker per warp, G = 32):
// the CTA streams the precision matrix through shared memory in tiles of `tr`
// rows (cp.async, double-buffered), so one read of P serves all its walkers
// instead of one per walker.  Each lane accumulates y = P v over the rows in the
// same order as lik_eval, so the result is the same to the bit.  Every thread of
// the CTA calls it (barriers inside); ptile holds 2 * tr * d_pad floats.
__device__ __forceinline__ void cp_async16(float *dst_smem, const float *src_gmem)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src_gmem) : "memory");
}

// NC consecutive floats at a 4 NC-byte aligned shared address, in one access
// (NC = 1, 2, 4): a warp then reads 32 NC consecutive floats without bank conflicts.
template <int NC>
__device__ __forceinline__ void vec_load(const float *p, float (&v)[NC])
{
    if constexpr (NC == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (NC == 2) {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        v[0] = q.x; v[1] = q.y;
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = p[c];
    }
}
template <int NC>
__device__ __forceinline__ void vec_store(float *p, const float (&v)[NC])
{
    if constexpr (NC == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (NC == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) p[c] = v[c];
    }
}

template <int KIND, int E>
__device__ float lik_dense_coop(const RunDesc &D, const ParView &P, const float (&x)[E], float (&g)[E], int c0,
                                float *rbuf, float *ptile, int tr)
{
    // Y[16][d_pad] = V[16][d] P as a register-blocked product: thread (wg, cg) accumulates
    // walkers 4 wg .. 4 wg + 3 by columns NC cg .. NC cg + NC - 1 (NC = d_pad / 128), so each
    // element of a P tile is read from shared memory by 4 threads instead of 16 warps.
    constexpr int NC = (E * 32) / 128;
    static_assert(NC >= 1 && NC <= 4 && NC * 128 == E * 32, "d_pad 128, 256 or 512");
    const int d = D.d, dp = D.d_pad;
    const bool mix = (KIND == NS_LIK_DENSE_MIX);
    // v to the walker's buffer (means in the lane-row layout; plain columns in rbuf)
#pragma unroll
    for (int h = 0; h < E / 4; ++h) {
        float4 v = make_float4(x[4 * h], x[4 * h + 1], x[4 * h + 2], x[4 * h + 3]);
        if (!mix) {
            const float4 mu = lane_quad<E>(P.means, threadIdx.x & 31, h);
            v.x -= mu.x; v.y -= mu.y; v.z -= mu.z; v.w -= mu.w;
        }
        const int c = c0 + 4 * h;
        if (c + 0 >= d) v.x = 0.f;
        if (c + 1 >= d) v.y = 0.f;
        if (c + 2 >= d) v.z = 0.f;
        if (c + 3 >= d) v.w = 0.f;
        reinterpret_cast<float4 *>(rbuf + c)[0] = v;
    }
    const int ntiles = (d + tr - 1) / tr;
    const int chunks_per_row = dp >> 2;
    auto load_tile = [&](int t, float *buf) {
        const int j0 = t * tr, jn = min(tr, d - j0);
        const int n = jn * chunks_per_row;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int jj = i / chunks_per_row, q = i - jj * chunks_per_row;
            cp_async16(buf + jj * dp + 4 * q, P.prec + (long)(j0 + jj) * dp + 4 * q);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    const int wg = threadIdx.x >> 7, cg = threadIdx.x & 127;
    const float *vrow = rbuf - (long)(threadIdx.x >> 5) * dp + (long)(4 * wg) * dp;  // V row of walker 4 wg
    float acc[4][NC];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[i][c] = 0.f;
    __syncthreads();  // every walker has staged v; the tiles of the previous call are no longer read
    load_tile(0, ptile);
    for (int t = 0; t < ntiles; ++t) {
        if (t + 1 < ntiles) {
            load_tile(t + 1, ptile + ((t + 1) & 1) * tr * dp);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const float *tb = ptile + (t & 1) * tr * dp + NC * cg;
        const int j0 = t * tr, jn = min(tr, d - j0);
        for (int jj = 0; jj < jn; ++jj) {
            float pv[NC];
            vec_load<NC>(tb + jj * dp, pv);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float vj = vrow[(long)i * dp + j0 + jj];
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[i][c] = fmaf(pv[c], vj, acc[i][c]);
            }
        }
        __syncthreads();  // the buffer of tile t is refilled by the load of tile t + 2
    }
    // Y through the tile buffer (16 x d_pad floats fit in 2 tr d_pad) in the lane-row
    // layout (NC columns never straddle a quad), then each walker reads its quads
#pragma unroll
    for (int i = 0; i < 4; ++i) vec_store<NC>(ptile + (long)(4 * wg + i) * dp + swz_col<E>(NC * cg), acc[i]);
    __syncthreads();
    float y[E];
    const float *yrow = ptile + (long)(threadIdx.x >> 5) * dp;
#pragma unroll
    for (int h = 0; h < E / 4; ++h) {
        const float4 t = lane_quad<E>(yrow, threadIdx.x & 31, h);
        y[4 * h] = t.x; y[4 * h + 1] = t.y; y[4 * h + 2] = t.z; y[4 * h + 3] = t.w;
    }
    return dense_finish<KIND, 32, E, true>(D, P, x, y, g, c0, nullptr);
}

// E consecutive floats of a lane (c0 a multiple of E, rows 16-byte aligned when E % 4 == 0):
// float4 accesses where E allows, so a warp moves its rows in E/4 wide instructions.
template <int E>
__device__ __forceinline__ void row_load(const float *src, float (&v)[E])
{
    if constexpr (E % 4 == 0) {
#pragma unroll
        for (int q = 0; q < E / 4; ++q) {
            const float4 t = reinterpret_cast<const float4 *>(src)[q];
            v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = src[e];
    }
}
template <int E>
__device__ __forceinline__ void row_store(float *dst, const float (&v)[E])
{
    if constexpr (E % 4 == 0) {
#pragma unroll
        for (int q = 0; q < E / 4; ++q)
            reinterpret_cast<float4 *>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) dst[e] = v[e];
    }
}

// The dense mixture after y = P x on the tensor-core walk (one walker per warp, means
// and P mu in the lane-row layout), for up to 8 components: the quadratic forms
// q_k = (x - mu_k).(y - P mu_k) of all components, their warp sums interleaved level by
// level (eight independent chains instead of one after another), then the log-sum-exp.
// Returns log L and, in r_lane, the responsibility r_k of component k = lane % 8; the
// score g = -(y - sum_k r_k P mu_k) (the r_k sum to one) is formed by mix_score8 only
// where a reflection needs it.
template <int E>
__device__ __forceinline__ float dense_mix_finish8(const RunDesc &D, const ParView &P, const float (&x)[E],
                                                   const float (&y)[E], float &r_lane)
{
    constexpr int KC = 8;
    const int K = D.n_comp;
    const int dp = D.d_pad;
    const int lane = threadIdx.x & 31;
    float q[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        q[k] = 0.f;
        if (k < K) {
            const float *mu = P.means + (long)k * dp;
            const float *pm = P.pmu + (long)k * dp;
#pragma unroll
            for (int h = 0; h < E / 4; ++h) {
                const float4 a = lane_quad<E>(mu, lane, h), b = lane_quad<E>(pm, lane, h);
                q[k] = fmaf(x[4 * h] - a.x, y[4 * h] - b.x, q[k]);
                q[k] = fmaf(x[4 * h + 1] - a.y, y[4 * h + 1] - b.y, q[k]);
                q[k] = fmaf(x[4 * h + 2] - a.z, y[4 * h + 2] - b.z, q[k]);
                q[k] = fmaf(x[4 * h + 3] - a.w, y[4 * h + 3] - b.w, q[k]);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < KC; ++k) q[k] += __shfl_xor_sync(0xffffffffu, q[k], o);
    }
    float m = -INFINITY;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        q[k] = (k < K) ? P.b[k] - 0.5f * q[k] : -INFINITY;  // t_k
        m = fmaxf(m, q[k]);
    }
    float s = 0.f, w_lane = 0.f;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const float w = (k < K) ? expf(q[k] - m) : 0.f;  // w_k
        s += w;
        if ((lane & 7) == k) w_lane = w;
    }
    r_lane = w_lane / s;
    return D.lik_const + m + logf(s);
}

// The score of the dense mixture from y (held in g) and the responsibilities (r_k in
// lane k of every eight): g = -y + sum_k r_k P mu_k.
template <int E>
__device__ __forceinline__ void mix_score8(const RunDesc &D, const ParView &P, float r_lane, float (&g)[E])
{
    const int K = D.n_comp;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int e = 0; e < E; ++e) g[e] = -g[e];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float rk = __shfl_sync(0xffffffffu, r_lane, k);
        if (k < K) {
            const float *pm = P.pmu + (long)k * D.d_pad;
#pragma unroll
            for (int h = 0; h < E / 4; ++h) {
                const float4 b = lane_quad<E>(pm, lane, h);
                g[4 * h] = fmaf(rk, b.x, g[4 * h]);
                g[4 * h + 1] = fmaf(rk, b.y, g[4 * h + 1]);
                g[4 * h + 2] = fmaf(rk, b.z, g[4 * h + 2]);
                g[4 * h + 3] = fmaf(rk, b.w, g[4 * h + 3]);
            }
        }
    }
}

// Dense likelihood of the 16 walkers of a CTA with the contraction on the tensor cores
// (ggns_tc.cuh); every thread of the CTA calls it.  `ok` turns false if a wait gave up.
// lazy: for the mixture of up to 8 components g holds y and r_lane the responsibilities
// on return, and mix_score8 forms the score when a reflection needs it; otherwise g is
// the score.
template <int KIND, int E, class Idle>
__device__ float lik_dense_tc(const RunDesc &D, const ParView &P, const float (&x)[E], float (&g)[E], int c0,
                              const tc::State &T, tc::Pipe &pp, bool &ok, float &r_lane, bool &lazy, const Idle &idle)
{
    const bool mix = (KIND == NS_LIK_DENSE_MIX);
    // v is staged in g (the score is written only after the contraction)
#pragma unroll
    for (int h = 0; h < E / 4; ++h) {
        float4 mu = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!mix) mu = lane_quad<E>(P.means, threadIdx.x & 31, h);
        const float m4[4] = {mu.x, mu.y, mu.z, mu.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = 4 * h + i;
            g[e] = (c0 + e < D.d) ? x[e] - m4[i] : 0.f;
        }
    }
    lazy = false;
    if constexpr (KIND == NS_LIK_DENSE_MIX) {
        if (D.n_comp <= 8) {
            ok = tc::contract<E>(T, pp, g, D.d_pad, D.tc_sv, D.tc_inv, g, idle);  // v is read before y is written
            lazy = true;
            return dense_mix_finish8<E>(D, P, x, g, r_lane);
        }
    }
    float y[E];
    ok = tc::contract<E>(T, pp, g, D.d_pad, D.tc_sv, D.tc_inv, y, idle);
    return dense_finish<KIND, 32, E, true>(D, P, x, y, g, c0, nullptr);
}

// ------------------------------------------------------------------------
// Prior draws (Algorithm 3, first step): x ~ U(box) from Philox purpose 0.
// One walker-tile group per point.
// ------------------------------------------------------------------------
template <int KIND, int G, int E>
__global__ void __launch_bounds__(HSS_THREADS) k_prior_init(DevCtx C, const int *run_list, int prec_in_smem)
{
    extern __shared__ float smem[];
    const int r = run_list[blockIdx.y];
    const RunDesc D = C.desc[r];
    const ParView P = load_params(C, D, smem, prec_in_smem);
    float *rbase = smem + param_smem_floats(D, prec_in_smem);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int lig = lane % G;
    const int grp = threadIdx.x / G;
    const int c0 = lig * E;
    const int groups_per_cta = HSS_THREADS / G;
    float *rbuf = rbase + (long)grp * D.d_pad;
    for (int base = blockIdx.x * groups_per_cta; base < D.n_live; base += gridDim.x * groups_per_cta) {
        const int i = base + grp;
        const bool act = i < D.n_live;
        const int ii = act ? i : 0;
        float x[E], g[E];
        if constexpr (E >= 4) {
#pragma unroll
            for (int b = 0; b < E / 4; ++b) {
                const U4 w = rng_block(D, 0, P_INIT, ii, 0, (c0 >> 2) + b);
                const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int c = c0 + 4 * b + t;
                    x[4 * b + t] = (c < D.d) ? fmaf(P.hi[c] - P.lo[c], u01(ws[t]), P.lo[c]) : 0.f;
                }
            }
        } else {
            const U4 w = rng_block(D, 0, P_INIT, ii, 0, c0 >> 2);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int c = c0 + e;
                x[e] = (c < D.d) ? fmaf(P.hi[c] - P.lo[c], u01(ws[c & 3]), P.lo[c]) : 0.f;
            }
        }
        const float ll = lik_eval<KIND, G, E>(D, P, x, g, c0, rbuf, nullptr);
        if (act) {
            float *dst = C.fa + D.x_off + (long)i * D.d_pad + c0;
#pragma unroll
            for (int e = 0; e < E; ++e) dst[e] = x[e];
            if (lig == 0) {
                C.logl[D.pt_off + i] = ll;
                C.label[D.pt_off + i] = 0;
            }
        }
    }
}

// ------------------------------------------------------------------------
// The reversible step (midpoint): the state the pick drew for walker w (now in its
// killed slot, flagged in wint[10]) is tested against L*; outside, the slot takes
// the walker's start point and its log L back (the slice-sampling rejection).
// One walker-tile group per walker.
// ------------------------------------------------------------------------
template <int KIND, int G, int E>
__global__ void __launch_bounds__(HSS_THREADS) k_eval_new(DevCtx C, const int *run_list, int prec_in_smem)
{
    extern __shared__ float smem[];
    const int r = run_list[blockIdx.y];
    const RunDesc D = C.desc[r];
    RunState *S = C.state + r;
    if (S->done || !D.midpoint) return;
    const ParView P = load_params(C, D, smem, prec_in_smem);
    float *rbase = smem + param_smem_floats(D, prec_in_smem);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int lig = lane % G;
    const int grp = threadIdx.x / G;
    const int c0 = lig * E;
    const int gpc = HSS_THREADS / G;
    const int dp = D.d_pad;
    float *rbuf = rbase + (long)grp * dp;
    const float lstar = static_cast<float>(S->lstar);
    for (int base = blockIdx.x * gpc; base < D.k; base += gridDim.x * gpc) {
        const int w = base + grp;
        const bool act = w < D.k;
        const int ww = act ? w : 0;
        int *flag = C.wint + (long)(D.w_off + ww) * WINT + 10;
        const bool need = act && *flag != 0;
        if (!__any_sync(0xffffffffu, need)) continue;  // the likelihood's group sums are warp-wide
        const int slot = C.order[D.pt_off + ww];
        float *xs = C.fa + D.x_off + (long)slot * dp + c0;
        float x[E], g[E];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = xs[e];
        const float ll = lik_eval<KIND, G, E>(D, P, x, g, c0, rbuf, nullptr);
        if (!need) continue;
        if (ll > lstar) {
            if (lig == 0) C.logl[D.pt_off + slot] = ll;
        } else {
            const int s0 = C.start_slot[D.w_off + ww];
            const float *src = C.fa + D.x_off + (long)s0 * dp + c0;
#pragma unroll
            for (int e = 0; e < E; ++e) xs[e] = src[e];
            if (lig == 0) {
                C.logl[D.pt_off + slot] = C.logl[D.pt_off + s0];
                C.wint[(long)(D.w_off + ww) * WINT + 6] = 1;
            }
        }
        if (lig == 0) *flag = 0;
    }
}

// ------------------------------------------------------------------------
// Batched Hamiltonian slice sampling (Algorithm 5), one of three phases:
//   phase 0: from the start point until the walker's own n_ref >= min_ref;
//            t_save = max over walkers of that step (the first step at which
//            min over walkers of n_ref >= min_ref).
//   phase 1: until t >= t_save, n_ref >= max_ref and t >= min_steps; saving
//            inside states from t_save on; t_stop = max over walkers.
//   phase 2: every walker continues to t_stop (the global stop), then emits
//            the reservoir pick into its killed slot.
// The three phases reproduce the global loop condition of Algorithm 5 without
// a grid-wide barrier: each walker's trajectory depends only on (seed, run,
// iteration, slot, step), so it can be cut at any step and resumed.
// ------------------------------------------------------------------------
template <int KIND, int G, int E>
__global__ void __launch_bounds__(HSS_THREADS) k_hss(DevCtx C, const int *run_list, int phase, int prec_in_smem)
{
    extern __shared__ float smem[];
    const int r = run_list[blockIdx.y];
    const RunDesc D = C.desc[r];
    RunState *S = C.state + r;
    if (S->done) return;
    // phase | 4: run only if the single-pass form of this iteration overflowed its records
    if (phase & 4) {
        if (!S->rec_overflow) return;
        phase &= 3;
    }
    const ParView P = load_params(C, D, smem, prec_in_smem);
    float *rbase = smem + param_smem_floats(D, prec_in_smem);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int lig = lane % G;
    const int gbase = lane - lig;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << gbase);
    const int grp = threadIdx.x / G;
    const int c0 = lig * E;
    float *rbuf = rbase + (long)grp * D.d_pad;
    const int W = D.k;
    const int dp = D.d_pad;
    const uint32_t iter = static_cast<uint32_t>(S->iter);
    const float dt = static_cast<float>(S->dt);
    const float lstar = static_cast<float>(S->lstar);
    const int t_save = (phase >= 1) ? S->t_save : 0x7fffffff;
    const int t_stop = (phase == 2) ? S->t_stop : 0;
    const float dlt = D.delta_p;
    const float keep = D.keep;

    float x[E], p[E], xr[E], g[E], eps[E], vmask[E];
#pragma unroll
    for (int e = 0; e < E; ++e) vmask[e] = (c0 + e < D.d) ? 1.f : 0.f;  // padded components keep p = 0
    int w = 0, t = 0, nref = 0, consec = 0, count = 0, nin = 0, nout = 0, nfold = 0;
    int res_start = 0;  // the reservoir holds a rejected (outside) step: emit the start point
    float res_ll = 0.f;
    bool active = false, exhausted = false;

    for (;;) {
        // ---- refill a finished group with the next walker of the run
        if (!active && !exhausted) {
            unsigned wid = 0;
            if (lig == 0) wid = atomicAdd(&S->wcount[phase], 1u);
            wid = __shfl_sync(gmask, wid, gbase);
            if (wid >= static_cast<unsigned>(W)) {
                exhausted = true;
            } else {
                w = static_cast<int>(wid);
                active = true;
                const int s0 = C.start_slot[D.w_off + w];
                if (phase == 0) {
                    const float *src = C.fa + D.x_off + (long)s0 * dp + c0;
#pragma unroll
                    for (int e = 0; e < E; ++e) x[e] = src[e];
                    lane_normals<E>(D, iter, P_MOM, w, 0, c0, p);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        if (c0 + e >= D.d) p[e] = 0.f;
                        xr[e] = x[e];
                    }
                    t = nref = consec = count = nin = nout = nfold = res_start = 0;
                    res_ll = 0.f;
                    // archive the dead point that this walker's output will replace
                    const int ks = C.order[D.pt_off + w];
                    const float *ksrc = C.fa + D.x_off + (long)ks * dp + c0;
                    const long drow = S->n_dead - W + w;
                    float *ddst = D.dead_x + (D.dead_off + drow) * dp + c0;
                    const bool din = gg_in(drow, D.dead_cap, S);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (din) ddst[e] = ksrc[e];
                } else {
                    const float *ws = C.fa + D.ws_off + (long)w * 3 * dp + c0;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        x[e] = ws[e];
                        p[e] = ws[dp + e];
                        xr[e] = ws[2 * dp + e];
                    }
                    const int *wi = C.wint + (D.w_off + w) * WINT;
                    t = wi[0]; nref = wi[1]; consec = wi[2]; count = wi[3]; nin = wi[4]; nout = wi[5];
                    res_start = wi[7];
                    nfold = wi[8];
                    res_ll = C.wres_logl[D.w_off + w];
                }
            }
        }
        // ---- stop test of the phase; finish the walker
        if (active) {
            bool stop;
            if (phase == 0) stop = (nref >= D.min_ref) || (t >= D.n_steps);
            else if (phase == 1) stop = (t >= t_save && nref >= D.max_ref && t >= D.min_steps) || (t >= D.n_steps);
            else stop = (t >= t_stop);
            if (stop) {
                if (phase < 2) {
                    float *ws = C.fa + D.ws_off + (long)w * 3 * dp + c0;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        ws[e] = x[e];
                        ws[dp + e] = p[e];
                        ws[2 * dp + e] = xr[e];
                    }
                    if (lig == 0) {
                        int *wi = C.wint + (D.w_off + w) * WINT;
                        wi[0] = t; wi[1] = nref; wi[2] = consec; wi[3] = count; wi[4] = nin; wi[5] = nout;
                        wi[7] = res_start;
                        wi[8] = nfold;
                        C.wres_logl[D.w_off + w] = res_ll;
                        if (phase == 0) atomicMax(&S->t_save, (nref >= D.min_ref) ? t : D.n_steps + 1);
                        else atomicMax(&S->t_stop, t);
                    }
                } else {
                    // emit: the reservoir pick, else (nothing saved, or a rejected outside
                    // step drawn) the start point
                    const int slot = C.order[D.pt_off + w];
                    float *dst = C.fa + D.x_off + (long)slot * dp + c0;
                    float out_ll;
                    if (count > 0 && !res_start) {
#pragma unroll
                        for (int e = 0; e < E; ++e) dst[e] = xr[e];
                        out_ll = res_ll;
                    } else {
                        const int s0 = C.start_slot[D.w_off + w];
                        const float *src = C.fa + D.x_off + (long)s0 * dp + c0;
#pragma unroll
                        for (int e = 0; e < E; ++e) dst[e] = src[e];
                        out_ll = C.logl[D.pt_off + s0];
                    }
                    if (lig == 0) {
                        C.logl[D.pt_off + slot] = out_ll;
                        C.label[D.pt_off + slot] = C.new_label[D.w_off + w];
                        atomicAdd(reinterpret_cast<unsigned long long *>(&S->n_in), static_cast<unsigned long long>(nin));
                        atomicAdd(reinterpret_cast<unsigned long long *>(&S->n_out), static_cast<unsigned long long>(nout));
                        if (nfold) atomicAdd(reinterpret_cast<unsigned long long *>(&S->n_fold), static_cast<unsigned long long>(nfold));
                        if (count == 0 || res_start) C.wint[(D.w_off + w) * WINT + 6] = 1;
                    }
                }
                active = false;
            }
        }
        __syncwarp();
        if (!__any_sync(0xffffffffu, active || !exhausted)) break;
        const bool stepping = active;

        // ---- one step of Algorithm 5 for every stepping walker of the warp
        const int ts = t + 1;
        // this step's random numbers depend only on (slot, step): draw them first
        uint32_t spare = 0;
        lane_normals<E>(D, iter, P_NOISE, w, ts, c0, eps, &spare);
        // the reservoir word: spare bits of the walker's noise block 0 (held by its lane 0)
        const uint32_t res_word = __shfl_sync(0xffffffffu, spare, gbase);
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = fmaf(p[e], dt, x[e]);
        wrap_periodic<KIND, E>(D, P, x, c0);
        const bool lfold = fold_box<KIND, E>(D, P, x, p, c0);
        const float ll = lik_eval<KIND, G, E>(D, P, x, g, c0, rbuf, nullptr);
        int outbox = 0;
        float nb[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            // padded components stay at 0 inside lo = hi = 0
            const int c = c0 + e;
            nb[e] = (x[e] < P.lo[c]) ? -1.f : ((x[e] > P.hi[c]) ? 1.f : 0.f);
            outbox += (nb[e] != 0.f);
        }
        // the box count and the fold flag (bit 16) in one group sum
        outbox = gsum_i<G>(outbox | (lfold ? 0x10000 : 0));
        const bool folded = (outbox >> 16) != 0;
        outbox &= 0xffff;
        const bool outside = (outbox > 0) || !(ll > lstar);
        float pnb = 0.f, pg = 0.f, gg = 0.f;
        if (__any_sync(0xffffffffu, stepping && outside)) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                pnb = fmaf(p[e], nb[e], pnb);
                pg = fmaf(p[e], g[e], pg);
                gg = fmaf(g[e], g[e], gg);
            }
            pnb = gsum<G>(pnb);
            pg = gsum<G>(pg);
            gg = gsum<G>(gg);
        }
        if (stepping && outside) {
            if (outbox > 0) {
                // reflect off the violated prior-box faces: n = nb / sqrt(#faces)
                const float c = __fdividef(2.f * pnb, static_cast<float>(outbox));
#pragma unroll
                for (int e = 0; e < E; ++e) p[e] = fmaf(-c, nb[e], p[e]);
            } else if (gg > 0.f && gg <= 3.0e38f) {
                // p' = p - 2 (p.n) n with n = g / |g|
                const float c = __fdividef(2.f * pg, gg);
#pragma unroll
                for (int e = 0; e < E; ++e) p[e] = fmaf(-c, g[e], p[e]);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) p[e] = -p[e];
            }
        }
        // momentum noise (with noise_inside, an outside step only reflects)
        if (stepping && !(outside && D.noise_inside)) {
            if (D.noise_mode == 1) {
#pragma unroll
                for (int e = 0; e < E; ++e) p[e] = fmaf(keep, p[e], dlt * eps[e] * vmask[e]);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) p[e] = p[e] * fmaf(dlt, eps[e], 1.f);
            }
        }
        if (stepping) {
            nref += outside ? 1 : 0;
            if (outside) { ++nout; ++consec; } else { ++nin; consec = 0; nfold += folded ? 1 : 0; }
        }
        // trajectory preservation: size-1 reservoir over the steps of the saving window
        // (inside steps only; with pick_all every step, a drawn outside step rejecting)
        const bool save = stepping && (!outside || D.pick_all) && (ts >= t_save);
        if (save) {
            ++count;
            if (D.keep_last || ((static_cast<uint64_t>(res_word) * static_cast<uint64_t>(count)) >> 32) == 0) {
                res_start = outside ? 1 : 0;
#pragma unroll
                for (int e = 0; e < E; ++e) xr[e] = x[e];
                res_ll = ll;
            }
        }
        // pruning: back to the start point with a fresh momentum
        if (stepping && D.prune_after > 0 && consec >= D.prune_after) {
            const int s0 = C.start_slot[D.w_off + w];
            const float *src = C.fa + D.x_off + (long)s0 * dp + c0;
#pragma unroll
            for (int e = 0; e < E; ++e) x[e] = src[e];
            lane_normals<E>(D, iter, P_PRUNE, w, ts, c0, p);
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (c0 + e >= D.d) p[e] = 0.f;
            consec = 0;
        }
        if (stepping) t = ts;
    }
}

// The momentum noise of step `step` drawn (Philox) and applied four components at a
// time, so that no array of normals stays live (E a multiple of 4); `add` false
// draws only the first block.  Returns the step's reservoir word (the spare bits of
// the lane's first block).  The same update as with the normals drawn ahead.
// The momentum noise of one step (all E normals of the lane and the reservoir word, the
// same Philox blocks and Box-Muller pairs as noise_in_place).
template <int E>
__device__ __forceinline__ uint32_t draw_noise(const RunDesc &D, uint32_t iter, uint32_t slot, uint32_t step, int c0,
                                               float (&z)[E])
{
    static_assert(E % 4 == 0, "whole Philox blocks");
    uint32_t word = 0;
#pragma unroll
    for (int b = 0; b < E / 4; ++b) {
        const U4 r = rng_block(D, iter, P_NOISE, slot, step, static_cast<uint32_t>((c0 >> 2) + b));
        if (b == 0) word = spare_bits(r);
        box_muller(r.x, r.y, z[4 * b], z[4 * b + 1]);
        box_muller(r.z, r.w, z[4 * b + 2], z[4 * b + 3]);
    }
    return word;
}

// p takes the noise z of the step, as noise_in_place applies it.
template <int E>
__device__ __forceinline__ void apply_noise(const RunDesc &D, int c0, float keep, float dlt, const float (&z)[E],
                                            float (&p)[E])
{
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (D.noise_mode == 1)
            p[e] = fmaf(keep, p[e], dlt * z[e] * ((c0 + e < D.d) ? 1.f : 0.f));
        else
            p[e] = p[e] * fmaf(dlt, z[e], 1.f);
    }
}

template <int E>
__device__ __forceinline__ uint32_t noise_in_place(const RunDesc &D, uint32_t iter, uint32_t slot, uint32_t step,
                                                   int c0, bool add, float keep, float dlt, float (&p)[E])
{
    static_assert(E % 4 == 0, "whole Philox blocks");
    uint32_t word = 0;
#pragma unroll
    for (int b = 0; b < E / 4; ++b) {
        if (b > 0 && !add) break;
        const U4 r = rng_block(D, iter, P_NOISE, slot, step, static_cast<uint32_t>((c0 >> 2) + b));
        if (b == 0) word = spare_bits(r);
        if (!add) break;
        float z[4];
        box_muller(r.x, r.y, z[0], z[1]);
        box_muller(r.z, r.w, z[2], z[3]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = 4 * b + i;
            if (D.noise_mode == 1)
                p[e] = fmaf(keep, p[e], dlt * z[i] * ((c0 + e < D.d) ? 1.f : 0.f));
            else
                p[e] = p[e] * fmaf(dlt, z[i], 1.f);
        }
    }
    return word;
}

// ------------------------------------------------------------------------
// Single-pass HSS (Algorithm 5) when every walker of the launch is resident.
// A walker steps, records each step (inside flag, reservoir word, log L and, for
// inside states, x), and registers with run-wide counters the step at which its
// own n_ref first reaches min_ref and the step at which it meets its stop rule
// (n_ref >= max_ref and t >= min_steps, or n_steps).  t_save and t_stop are the
// maxima of those steps, i.e. the first steps at which min over walkers of n_ref
// reaches min_ref and max_ref.  A walker stops once every walker has registered
// and it has reached t_stop; steps it took beyond t_stop are discarded.  Because
// a trajectory depends only on (seed, run, iteration, slot, step), the result
// equals the three-phase form exactly.  k_hss_pick then replays the reservoir
// over the recorded window [t_save, t_stop].  A walker that reaches the record
// length before the run's stop is known sets rec_overflow; the three-phase
// kernels then redo the iteration.
// Records of walker w: meta[(w * rec_len + t - 1)] = (word, flags), ll[...] = log L,
// x[(w * rec_len + t - 1) * xs + c] (inside steps only), rows offset by the run's rec_base.
// ------------------------------------------------------------------------

// COOP: dense kinds whose precision matrix does not fit in shared memory; one
// walker per warp, COOP_THREADS / 32 walkers per CTA stepping together, each CTA
// taking a fixed block of walkers, the likelihood from lik_dense_coop with P
// tiles of coop_tr rows.  Same trajectories as the form with one walker group
// per refill.
constexpr int COOP_THREADS = 512;

// TC (with COOP): the contraction of the cooperative walk on the tensor cores.
template <int KIND, int G, int E, bool COOP = false, bool TC = false>
__global__ void __launch_bounds__(COOP ? COOP_THREADS : HSS_THREADS, COOP ? 1 : ((E >= 16) ? 2 : 4))
    k_hss1(DevCtx C, const int *run_list, RecView R, const long *rec_base, int prec_in_smem, int coop_tr)
{
    static_assert(!COOP || G == 32, "one walker per warp");
    static_assert(!TC || (COOP && COOP_THREADS == 32 * tc::WALKERS), "the tensor-core walk is the 16-warp CTA form");
    extern __shared__ float smem[];
    const int r = run_list[blockIdx.y];
    // the cooperative walk keeps the run's descriptor and parameter view in shared
    // memory (read there when used) to leave its registers to the walker
    __shared__ RunDesc sD;
    __shared__ ParView sP;
    RunDesc Dl;
    if constexpr (COOP) {
        if (threadIdx.x == 0) sD = C.desc[r];
        __syncthreads();
    } else {
        Dl = C.desc[r];
    }
    const RunDesc &D = COOP ? sD : Dl;
    RunState *S = C.state + r;
    if (S->done) return;
    const ParView Pl = load_params(C, D, smem, prec_in_smem);
    if constexpr (COOP) {
        if (threadIdx.x == 0) sP = Pl;
    }
    float *rbase = smem + param_smem_floats(D, prec_in_smem);
    __syncthreads();
    const ParView &P = COOP ? sP : Pl;
    if constexpr (COOP) {
        // the box, the means and P mu into the lane-row layout (read as quads below)
        const ParLayout PL = par_layout(D.d, D.d_pad, D.n_comp, D.kind);
        swizzle_rows<E>(smem + PL.lo, 2 + comp_slots(D.n_comp, D.kind), D.d_pad);
        if (P.pmu) swizzle_rows<E>(const_cast<float *>(P.pmu), D.n_comp, D.d_pad);
        __syncthreads();
    }
    const long rb = rec_base[r];  // first record row of this run
    const int nsteps = (D.d_pad & 3) ? 0 : noise_steps(R.nT, S->t_stop_last);
    const long nrow0 = (rb / R.rec_len) * R.nT;  // first noise row of this run
    const int lane = threadIdx.x & 31;
    const int lig = lane % G;
    const int gbase = lane - lig;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << gbase);
    const int grp = threadIdx.x / G;
    const int c0 = lig * E;
    float *rbuf = rbase + (long)grp * D.d_pad;
    const int W = D.k;
    const int dp = D.d_pad;
    const int L = min(R.rec_len, D.n_steps);
    // COOP: the P tiles follow the walkers' buffers (16-byte aligned)
    float *ptile = nullptr;
    if constexpr (COOP) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(rbase + (long)(blockDim.x / 32) * dp);
        ptile = reinterpret_cast<float *>((a + 15) & ~uintptr_t(15));
    }
    bool coop_first = true;
    (void)coop_first;
    (void)coop_tr;
    __shared__ int s_tc_fail;
    __shared__ tc::State T;
    tc::Pipe tc_pipe;
    bool tc_ok = true;
    float tc_r = 0.f;      // responsibility of component lane % 8 (tensor-core mixture walk)
    bool tc_lazy = false;  // g holds y until the score is needed
    __shared__ uint32_t s_nz_word[COOP_THREADS / 32];  // reservoir words of the stashed noise
    __shared__ int s_nz_act[COOP_THREADS / 32];        // walkers stepping this loop round
    int loop_i = 0;                                    // loop rounds so far (= t of the active walkers)
    if constexpr (TC) {
        // a CTA without walkers of this run leaves before it takes tensor memory
        if (static_cast<long>(blockIdx.x) * (blockDim.x / 32) >= W) return;
        const uintptr_t a = reinterpret_cast<uintptr_t>(rbase);
        tc::setup(T, reinterpret_cast<char *>((a + 1023) & ~uintptr_t(1023)), P.ptc, dp, &s_tc_fail);
    }
    (void)tc_ok;
    const uint32_t iter = static_cast<uint32_t>(S->iter);
    const float dt = static_cast<float>(S->dt);
    const float lstar = static_cast<float>(S->lstar);
    const float dlt = D.delta_p;
    const float keep = D.keep;
    volatile int *v_remain = &S->remain_max;
    volatile int *v_tstop = &S->t_stop1;

    // eps: the momentum noise of a step.  The cooperative walk draws it where it is
    // used (Philox on the ALUs; nothing stays live across the step); the other walks
    // load or draw it once the previous step is done, so that the load completes
    // while the coming step runs.
    float x[E], p[E], g[E], eps[E];
    int w = 0, t = 0, nref = 0, consec = 0;
    bool reg_min = false, reg_max = false;
    bool active = false, exhausted = false;
    // walkers still to register (read one step ahead, the same value in every lane
    // of a group: one load instruction) and, once that reached 0, the final t_stop
    int rem_seen = 1, tstop_final = -1;
    // this walker's record rows
    uint2 *rec_meta = nullptr;
    float *rec_ll = nullptr, *rec_x = nullptr;
    // noise of the next step (it depends only on slot and step, so it is drawn a
    // step ahead, beside the current step's likelihood)
    uint32_t spare = 0;

    for (;;) {
        if (!active && !exhausted) {
            unsigned wid = 0;
            if constexpr (COOP) {
                // a fixed walker per warp, taken once
                wid = coop_first ? static_cast<unsigned>(blockIdx.x * (blockDim.x / 32) + grp) : static_cast<unsigned>(W);
                coop_first = false;
            } else {
                if (lig == 0) wid = atomicAdd(&S->wcount1, 1u);
                wid = __shfl_sync(gmask, wid, gbase);
            }
            if (wid >= static_cast<unsigned>(W)) {
                exhausted = true;
            } else {
                w = static_cast<int>(wid);
                active = true;
                const int s0 = C.start_slot[D.w_off + w];
                const float *src = C.fa + D.x_off + (long)s0 * dp + c0;
#pragma unroll
                for (int e = 0; e < E; ++e) x[e] = src[e];
                lane_normals<E>(D, iter, P_MOM, w, 0, c0, p);
#pragma unroll
                for (int e = 0; e < E; ++e) p[e] = (c0 + e < D.d) ? p[e] : 0.f;
                if constexpr (!COOP) {
                    if (nsteps >= 1) {
                        const long nr0 = nrow0 + (long)w * R.nT;
                        row_load<E>(R.nz + nr0 * R.xs + c0, eps);
                        spare = R.nsp[nr0];
                    } else {
                        lane_normals<E>(D, iter, P_NOISE, w, 1, c0, eps, &spare);
                    }
                }
                t = nref = consec = 0;
                rem_seen = 1;
                tstop_final = -1;
                const long row0 = rb + (long)w * R.rec_len;
                rec_meta = R.meta + row0;
                rec_ll = R.ll + row0;
                rec_x = R.x + row0 * R.xs + c0;
                // archive the dead point that this walker's output will replace
                const int ks = C.order[D.pt_off + w];
                const float *ksrc = C.fa + D.x_off + (long)ks * dp + c0;
                const long drow = S->n_dead - W + w;
                float *ddst = D.dead_x + (D.dead_off + drow) * dp + c0;
                const bool din = gg_in(drow, D.dead_cap, S);
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (din) ddst[e] = ksrc[e];
                // a rule already met before the first step registers at t = 0
                reg_min = (D.min_ref == 0);
                reg_max = (D.max_ref == 0 && D.min_steps <= 0);
                if (lig == 0) {
                    if (reg_min) atomicSub(&S->remain_min, 1);
                    if (reg_max) {
                        __threadfence();
                        atomicSub(&S->remain_max, 1);
                    }
                }
            }
        }
        if (active) {
            // stop once every walker has met its stop rule and this one has reached t_stop,
            // or at the record length / step cap (every lane of the group decides alike)
            if (reg_max && rem_seen == 0 && tstop_final < 0) {
                // every walker has registered: t_stop is final (read after the count)
                __threadfence();
                tstop_final = *v_tstop;
            }
            const bool at_stop = tstop_final >= 0 && t >= tstop_final;
            if (t >= L && !at_stop && L < D.n_steps && lig == 0) {
                // the stop may not be known yet: decide on fresh values
                const int rem_now = *v_remain;
                __threadfence();
                if (!(reg_max && rem_now == 0 && t >= *v_tstop)) S->rec_overflow = 1;
            }
            if (at_stop || t >= L) active = false;
        }
        if constexpr (COOP) {
            if constexpr (TC) {
                if (lane == 0) s_nz_act[grp] = active ? 1 : 0;
            }
            if (!__syncthreads_or(active)) break;
            if constexpr (TC) {
                if (s_tc_fail) {
                    if (threadIdx.x == 0) S->status = NS_ERR_TIMEOUT;
                    break;
                }
            }
        } else {
            if (!__any_sync(0xffffffffu, active || !exhausted)) break;
        }
        const bool stepping = active;
        // the registration count for the next stop test, read while this step runs
        if (stepping && reg_max && rem_seen != 0) rem_seen = *v_remain;

        // ---- one step of Algorithm 5 (as in k_hss); with midpoint the time-reversible
        // form: half move, the evaluation and the reflection at the half step, half move
        const int ts = t + 1;
        uint32_t res_word = 0;
        if constexpr (!COOP) res_word = __shfl_sync(0xffffffffu, spare, gbase);
        const float hdt = D.midpoint ? 0.5f * dt : dt;
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = fmaf(p[e], hdt, x[e]);
        wrap_periodic<KIND, E>(D, P, x, c0);
        const bool lfold = fold_box<KIND, E, COOP>(D, P, x, p, c0);
        float ll;
        if constexpr (TC) {
            // the warps without a pipeline role (warps STAGES + 1 ..) draw this step's
            // momentum noise while P streams, their own and that of the warps with a role,
            // and keep it in the walker's tensor-memory columns (the reservoir word in shared
            // memory) until the step applies it.  Warp n's columns lie in the lanes of
            // quarter n % 4, so the i-th role warp of a quarter is served by the (i mod h)-th
            // idle warp of that quarter (h of them).  Active walkers of a CTA step in
            // lock-step from t = 0: the step of every active walker is the loop count + 1.
            auto idle = [&]() {
                const int nw = static_cast<int>(blockDim.x >> 5);
                const int q = grp & 3;
                const int h0 = tc::STAGES + 1 + ((q - (tc::STAGES + 1)) % 4 + 4) % 4;  // first idle warp of quarter q
                const int nh = (nw - 1 - h0) / 4 + 1;
                const int mine = (grp - h0) / 4;
                for (int i = -1, n = grp; n >= 0;) {
                    if (s_nz_act[n]) {
                        const uint32_t slot = static_cast<uint32_t>(blockIdx.x * nw + n);
                        float z[E];
                        const uint32_t wd = draw_noise<E>(D, iter, slot, static_cast<uint32_t>(loop_i + 1), c0, z);
                        tc::tmem_store<E>(tc::noise_addr(T, n), z);
                        if (lane == 0) s_nz_word[n] = wd;
                    }
                    // the next role warp of quarter q served by this warp
                    for (n = -1, ++i; q + 4 * i <= tc::STAGES; ++i) {
                        if (i % nh == mine) {
                            n = q + 4 * i;
                            break;
                        }
                    }
                }
            };
            ll = lik_dense_tc<KIND, E>(D, P, x, g, c0, T, tc_pipe, tc_ok, tc_r, tc_lazy, idle);
        } else if constexpr (COOP) {
            ll = lik_dense_coop<KIND, E>(D, P, x, g, c0, rbuf, ptile, coop_tr);
        } else {
            ll = lik_eval<KIND, G, E>(D, P, x, g, c0, rbuf, nullptr);
        }
        // the box normal n_e in {-1, 0, 1} (recomputed below for a reflection off the box);
        // the reflection's group sums are reduced together with the box count: four
        // independent trees instead of two in sequence behind a vote (same sums)
        int outbox = 0;
        float pnb = 0.f, pg = 0.f, gg = 0.f;
        if constexpr (COOP) {
#pragma unroll
            for (int h = 0; h < E / 4; ++h) {
                const float4 lo4 = lane_quad<E>(P.lo, lane, h), hi4 = lane_quad<E>(P.hi, lane, h);
                const float lo[4] = {lo4.x, lo4.y, lo4.z, lo4.w}, hi[4] = {hi4.x, hi4.y, hi4.z, hi4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int e = 4 * h + i;
                    const float nb = (x[e] < lo[i]) ? -1.f : ((x[e] > hi[i]) ? 1.f : 0.f);
                    outbox += (nb != 0.f);
                    pnb = fmaf(p[e], nb, pnb);
                }
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int c = c0 + e;
                const float nb = (x[e] < P.lo[c]) ? -1.f : ((x[e] > P.hi[c]) ? 1.f : 0.f);
                outbox += (nb != 0.f);
                pnb = fmaf(p[e], nb, pnb);
            }
        }
        // the score enters only a reflection off the iso-likelihood contour; the tensor-core
        // walk (one walker per warp: the test is uniform over the warp) skips it on the
        // other steps
        bool need_g = true;
        if constexpr (TC) {
            need_g = !(ll > lstar);
            if (need_g && tc_lazy) mix_score8<E>(D, P, tc_r, g);
        }
        if (need_g) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                pg = fmaf(p[e], g[e], pg);
                gg = fmaf(g[e], g[e], gg);
            }
        }
        // the box count and the fold flag (bit 16) in one group sum
        outbox = gsum_i<G>(outbox | (lfold ? 0x10000 : 0));
        const bool folded = (outbox >> 16) != 0;
        outbox &= 0xffff;
        pnb = gsum<G>(pnb);
        if (need_g) {
            pg = gsum<G>(pg);
            gg = gsum<G>(gg);
        }
        const bool outside = (outbox > 0) || !(ll > lstar);
        if (stepping && outside) {
            if (outbox > 0) {
                const float cc = __fdividef(2.f * pnb, static_cast<float>(outbox));
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int c = COOP ? swz_col<E>(c0 + e) : c0 + e;
                    const float nb = (x[e] < P.lo[c]) ? -1.f : ((x[e] > P.hi[c]) ? 1.f : 0.f);
                    p[e] = fmaf(-cc, nb, p[e]);
                }
            } else if (gg > 0.f && gg <= 3.0e38f) {
                const float cc = __fdividef(2.f * pg, gg);
#pragma unroll
                for (int e = 0; e < E; ++e) p[e] = fmaf(-cc, g[e], p[e]);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) p[e] = -p[e];
            }
        }
        bool folded_all = folded;
        if (D.midpoint) {
            // the second half move to the step's state (the box reflects it exactly too)
#pragma unroll
            for (int e = 0; e < E; ++e) x[e] = fmaf(p[e], hdt, x[e]);
            const bool lfold2 = fold_box<KIND, E, COOP>(D, P, x, p, c0);
            // every lane takes the group sum (the groups of a warp differ in `folded`)
            const int nf2 = gsum_i<G>(lfold2 ? 1 : 0);
            folded_all = folded || nf2 != 0;
        }
        if (stepping) {
            // momentum noise (with noise_inside, an outside step only reflects; with midpoint
            // every state takes the refresh)
            const bool add_noise = D.midpoint || !(outside && D.noise_inside);
            if constexpr (COOP) {
                // one walker per warp: `stepping` is uniform over the warp
                if constexpr (TC) {
                    // drawn during the contraction (published by its barriers)
                    spare = s_nz_word[grp];
                    if (add_noise) {
                        float z[E];
                        tc::fence_after_sync();
                        tc::tmem_load<E>(tc::noise_addr(T, grp), z);
                        apply_noise<E>(D, c0, keep, dlt, z, p);
                    }
                } else {
                    spare = noise_in_place<E>(D, iter, w, ts, c0, add_noise, keep, dlt, p);
                }
                res_word = __shfl_sync(0xffffffffu, spare, 0);
            } else if (add_noise) {
                if (D.noise_mode == 1) {
#pragma unroll
                    for (int e = 0; e < E; ++e) p[e] = fmaf(keep, p[e], dlt * eps[e] * ((c0 + e < D.d) ? 1.f : 0.f));
                } else {
#pragma unroll
                    for (int e = 0; e < E; ++e) p[e] = p[e] * fmaf(dlt, eps[e], 1.f);
                }
            }
            // the next step's noise
            if constexpr (!COOP) {
                if (ts + 1 <= nsteps) {
                    const long nr1 = nrow0 + (long)w * R.nT + ts;
                    row_load<E>(R.nz + nr1 * R.xs + c0, eps);
                    spare = R.nsp[nr1];
                } else {
                    lane_normals<E>(D, iter, P_NOISE, w, ts + 1, c0, eps, &spare);
                }
            }
            nref += outside ? 1 : 0;
            consec = outside ? consec + 1 : 0;
            // record the step (row t of this walker's rec_len rows): x of the inside steps, of
            // every step with midpoint (its state, which the pick may draw)
            const bool rin = gg_in(t, R.rec_len, S);
            if ((!outside || D.midpoint) && rin) row_store<E>(rec_x, x);
            if (lig == 0 && rin) {
                // flags: bit 0 outside, bit 1 an inside step on which the box reflected the walker
                *rec_meta = make_uint2(res_word, outside ? 1u : (folded_all ? 2u : 0u));
                *rec_ll = ll;
            }
            rec_x += R.xs;
            ++rec_meta;
            ++rec_ll;
            const bool reg_min_now = !reg_min && (nref >= D.min_ref || ts >= D.n_steps);
            const bool reg_max_now = !reg_max && ((nref >= D.max_ref && ts >= D.min_steps) || ts >= D.n_steps);
            if (lig == 0 && (reg_min_now || reg_max_now)) {
                if (reg_min_now) {
                    atomicMax(&S->t_save1, (nref >= D.min_ref) ? ts : D.n_steps + 1);
                    __threadfence();
                    atomicSub(&S->remain_min, 1);
                }
                if (reg_max_now) {
                    atomicMax(&S->t_stop1, ts);
                    __threadfence();
                    atomicSub(&S->remain_max, 1);
                }
            }
            reg_min = reg_min || nref >= D.min_ref || ts >= D.n_steps;
            reg_max = reg_max || (nref >= D.max_ref && ts >= D.min_steps) || ts >= D.n_steps;
            // pruning: back to the start point with a fresh momentum
            if (D.prune_after > 0 && consec >= D.prune_after) {
                const int s0 = C.start_slot[D.w_off + w];
                const float *src = C.fa + D.x_off + (long)s0 * dp + c0;
#pragma unroll
                for (int e = 0; e < E; ++e) x[e] = src[e];
                lane_normals<E>(D, iter, P_PRUNE, w, ts, c0, p);
#pragma unroll
                for (int e = 0; e < E; ++e) p[e] = (c0 + e < D.d) ? p[e] : 0.f;
                consec = 0;
            }
            t = ts;
        }
        if constexpr (TC) ++loop_i;
    }
    if constexpr (TC) tc::teardown(T, tc_pipe);
}

// ------------------------------------------------------------------------
// ns_lik_forward / ns_lik_backward on caller points x[n][d] (unpadded).
// mode 0: forward (logl, grad);  mode 1: adjoint (gx = gout * grad, gmu += ...)
// ------------------------------------------------------------------------
template <int KIND, int G, int E>
__global__ void __launch_bounds__(HSS_THREADS) k_lik_points(DevCtx C, int run, const float *xin, long n, int mode,
                                                           float *logl, float *grad, const float *gout,
                                                           float *gmu, int prec_in_smem)
{
    extern __shared__ float smem[];
    const RunDesc D = C.desc[run];
    const ParView P = load_params(C, D, smem, prec_in_smem);
    float *rbase = smem + param_smem_floats(D, prec_in_smem);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int lig = lane % G;
    const int grp = threadIdx.x / G;
    const int c0 = lig * E;
    const int gpc = HSS_THREADS / G;
    float *rbuf = rbase + (long)grp * D.d_pad;
    float resp[KMAX_COMP];
    for (long base = (long)blockIdx.x * gpc; base < n; base += (long)gridDim.x * gpc) {
        const long i = base + grp;
        const bool act = i < n;
        const long ii = act ? i : 0;
        float x[E], g[E];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = (c0 + e < D.d) ? xin[ii * D.d + c0 + e] : 0.f;
        const bool want_mu = (mode == 1) && gmu != nullptr && kind_has_means(KIND);
        const float ll = lik_eval<KIND, G, E>(D, P, x, g, c0, rbuf, want_mu ? resp : nullptr);
        if (!act) continue;
        if (mode == 0) {
            if (lig == 0) logl[i] = ll;
            if (grad) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (c0 + e < D.d) grad[i * D.d + c0 + e] = g[e];
            }
        } else {
            const float go = gout[i];
            if (grad) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (c0 + e < D.d) grad[i * D.d + c0 + e] = go * g[e];
            }
            if (want_mu) {
                const int K = (KIND == NS_LIK_ISO_GAUSS || KIND == NS_LIK_DENSE_GAUSS) ? 1 : D.n_comp;
                if constexpr (KIND == NS_LIK_DENSE_MIX) {
                    // the mixture shares P and the responsibilities sum to one, so the score
                    // -g = y - sum_k resp_k P mu_k gives y = P x back without a second product
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        float t = -g[e];
                        for (int k = 0; k < K; ++k) t = fmaf(resp[k], P.pmu[(long)k * D.d_pad + c0 + e], t);
                        g[e] = t;
                    }
                }
                for (int k = 0; k < K; ++k) {
                    const float rk = (KIND == NS_LIK_ISO_GAUSS || KIND == NS_LIK_DENSE_GAUSS) ? 1.f : resp[k];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int c = c0 + e;
                        if (c >= D.d) continue;
                        float v;
                        if (KIND == NS_LIK_ISO_GAUSS || KIND == NS_LIK_MIX_ISO) {
                            v = P.a[k] * (x[e] - P.means[(long)k * D.d_pad + c]);
                        } else if (KIND == NS_LIK_DENSE_GAUSS) {
                            v = -g[e];  // P (x - mu)
                        } else {
                            v = g[e] - P.pmu[(long)k * D.d_pad + c];  // P (x - mu_k) = y - P mu_k
                        }
                        atomicAdd(&gmu[(long)k * D.d + c], go * rk * v);
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------------------
// Posterior-weighted parameter gradient over the dead arena (partials).
// part[blk][K][d] (FP64) += sum_i p_i resp_ik v_ik, p_i = exp(logw_i + logL_i - logZ).
// Dead points with p_i < e^-60 are skipped (warps whose points all fall below it skip
// the likelihood): together they move the sum by less than n_dead e^-60 max |v|, far
// below its FP64 rounding.  For the dense mixture v_ik = P (x_i - mu_k) = y_i - P mu_k
// comes from the score the likelihood returns, -g_i = y_i - sum_j resp_ij P mu_j, so
// y_i = P x_i is formed once per point, not once per component.
// ------------------------------------------------------------------------
template <int KIND, int G, int E>
__global__ void __launch_bounds__(HSS_THREADS) k_grad_means(DevCtx C, int run, double logz, double *part,
                                                           int prec_in_smem)
{
    extern __shared__ float smem[];
    const RunDesc D = C.desc[run];
    const RunState *S = C.state + run;
    const ParView P = load_params(C, D, smem, prec_in_smem);
    float *rbase = smem + param_smem_floats(D, prec_in_smem);
    double *acc = reinterpret_cast<double *>(rbase + (long)(HSS_THREADS / G) * D.d_pad + 4);
    acc = reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(acc) + 15) & ~uintptr_t(15));
    const int K = (KIND == NS_LIK_ISO_GAUSS || KIND == NS_LIK_DENSE_GAUSS) ? 1 : D.n_comp;
    for (int i = threadIdx.x; i < K * D.d; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int lig = lane % G;
    const int grp = threadIdx.x / G;
    const int c0 = lig * E;
    const int gpc = HSS_THREADS / G;
    float *rbuf = rbase + (long)grp * D.d_pad;
    float resp[KMAX_COMP];
    const long n = S->n_dead;
    for (long base = (long)blockIdx.x * gpc; base < n; base += (long)gridDim.x * gpc) {
        const long i = base + grp;
        const bool act = i < n && gg_in(i, D.dead_cap, C.state + run);
        const long ii = act ? i : 0;
        const double lp = act ? (D.dead_logw[D.dead_off + ii] + (double)D.dead_logl[D.dead_off + ii] - logz)
                              : -INFINITY;
        const bool keep = lp > -60.0;
        if (!__any_sync(0xffffffffu, keep)) continue;  // the likelihood's group sums are warp-wide
        const float *src = D.dead_x + (D.dead_off + ii) * D.d_pad + c0;
        float x[E], g[E];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = src[e];
        lik_eval<KIND, G, E>(D, P, x, g, c0, rbuf, resp);
        if (!keep) continue;
        const double pw = exp(lp);
        if constexpr (KIND == NS_LIK_DENSE_MIX) {
            // y - sum_j resp_j P mu_j = -g; add the weighted P mu back once
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int c = c0 + e;
                float t = -g[e];
                for (int k = 0; k < K; ++k) t = fmaf(resp[k], P.pmu[(long)k * D.d_pad + c], t);
                g[e] = t;  // y
            }
        }
        for (int k = 0; k < K; ++k) {
            const float rk = (KIND == NS_LIK_ISO_GAUSS || KIND == NS_LIK_DENSE_GAUSS) ? 1.f : resp[k];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int c = c0 + e;
                if (c >= D.d) continue;
                float v;
                if (KIND == NS_LIK_ISO_GAUSS || KIND == NS_LIK_MIX_ISO) {
                    v = P.a[k] * (x[e] - P.means[(long)k * D.d_pad + c]);
                } else if (KIND == NS_LIK_DENSE_GAUSS) {
                    v = -g[e];
                } else {
                    v = g[e] - P.pmu[(long)k * D.d_pad + c];
                }
                atomicAdd(&acc[k * D.d + c], pw * (double)rk * (double)v);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < K * D.d; i += blockDim.x) part[(long)blockIdx.x * K * D.d + i] = acc[i];
}

}  // namespace ggns
