// ggns_iter.cu -- per-iteration kernels that are not specialised on the
// likelihood: lowest-likelihood selection, the FP64 evidence statistics of
// Appendix H, spawning, k-NN cluster finding (Algorithm 4), the iteration tail
// (step-size rule and termination of Algorithm 3), the final sweep, and the
// component entry points built on them.
#include <cstdio>

#include "ggns_iter.cuh"

namespace ggns {

// ------------------------------------------------------------------------
// Block-wide bitonic sort of npow2 64-bit keys in shared memory (ascending).
// ------------------------------------------------------------------------
// Ascending bitonic sort of npow2 keys in shared memory by the whole block.
// Stages whose partner distance j is at least 32 exchange through shared memory
// (one barrier each); the stages with j < 32 of each merge run in registers with
// warp shuffles: element i = tid + m * blockDim and its partner i ^ j sit in the
// same warp at the same m.  blockDim is a multiple of 32.
__device__ __forceinline__ unsigned long long bitonic_shfl_step(unsigned long long v, int i, int j, int k)
{
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
    const bool up = (i & k) == 0;     // ascending block of the merge
    const bool lower = (i & j) == 0;  // this element takes the smaller key when ascending
    const bool take_min = (up == lower);
    return take_min ? (o < v ? o : v) : (o > v ? o : v);
}

__device__ void bitonic_warp_stages(unsigned long long *keys, int npow2, int k, int j_top)
{
    // stages j = j_top, j_top / 2, ..., 1 of the merge of size k, in registers
    for (int i0 = 0; i0 < npow2; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        if (i0 + (int)(threadIdx.x & ~31u) >= npow2) continue;  // whole warp past the keys
        unsigned long long v = keys[i];
        for (int j = j_top; j > 0; j >>= 1) v = bitonic_shfl_step(v, i, j, k);
        keys[i] = v;
    }
}

__device__ void block_bitonic_sort(unsigned long long *keys, int npow2)
{
    if (npow2 < 32) {
        for (int k = 2; k <= npow2; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const unsigned long long a = keys[i], b = keys[ixj];
                        const bool up = (i & k) == 0;
                        if ((a > b) == up) {
                            keys[i] = b;
                            keys[ixj] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        return;
    }
    // merges of size 2 .. 32: all stages inside a warp
    for (int i0 = 0; i0 < npow2; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        if (i0 + (int)(threadIdx.x & ~31u) >= npow2) continue;
        unsigned long long v = keys[i];
        for (int k = 2; k <= 32; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) v = bitonic_shfl_step(v, i, j, k);
        keys[i] = v;
    }
    __syncthreads();
    for (int k = 64; k <= npow2; k <<= 1) {
        for (int j = k >> 1; j >= 32; j >>= 1) {
            for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = keys[i], b = keys[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
        bitonic_warp_stages(keys, npow2, k, 16);
        __syncthreads();
    }
}

__host__ __device__ __forceinline__ int next_pow2(int n)
{
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

// Key buffer: npow2 64-bit keys, reused for the kill arrays (12 bytes per kill).
__host__ __device__ __forceinline__ size_t key_region_bytes(int n)
{
    const size_t a = (size_t)next_pow2(n) * 8, b = (size_t)n * 12;
    return ((a > b ? a : b) + 15) & ~size_t(15);
}

// ------------------------------------------------------------------------
// Appendix H statistics for a batch of kills, in closed form.
//
// The kills j = 0..k-1 arrive in ascending log L order with cluster labels
// p_j.  Because update2/8/9 only rescale by n/(n+1) and n/(n+2), the volume
// moments after r kills of a cluster telescope:
//     X_c -> X_c (n_c - r + 1)/(n_c + 1),
//     X_c^2 -> X_c^2 (n_c - r + 1)(n_c - r + 2)/((n_c + 1)(n_c + 2)),
// and every kill of cluster c receives the prior mass X_c / (n_c + 1) of the
// statistics at the start of the batch.  Writing ZX_c = X_c zeta_c, the
// updates update5/6/7 add to zeta a constant multiple of L_j per kill, so
// update3 becomes a sum over ordered pairs i < j.  With l_j = exp(L_j - L_ref):
//   S1_c = sum_{j in c} l_j,  S2_c = sum_{j in c} l_j^2,
//   U_c  = sum_{j in c} l_j sum_{i<j, i in c} l_i,
//   V_c  = sum_{j in c} l_j sum_{i<j} a_{c,p_i} l_i,  a_{c,c} = X2_c/((n_c+2) X_c),
//          a_{c,q} = XX_qc/((n_q+1) X_c)   (scaled by 1/X_ref to stay in range),
// the batch applies exactly the same moments as the sequential update0-9.
// One CTA per run; each of the first 256 threads owns a contiguous chunk of
// kills, chunk sums are combined with sequential (deterministic) scans.
// ------------------------------------------------------------------------
constexpr int EV_THREADS = 256;
constexpr int EV_CB = 8;  // target clusters per pass

struct EvScratch {
    double wtot[EV_CB][EV_THREADS / 32];
    double coef[EV_CB][CMAX];
    double S1[CMAX], S2[CMAX], U[CMAX], V[CMAX];
    // per-cluster logs: lg = {log(n+1), log(n+2), log(r+1), log(r+2)} with r = n - m (-inf when r <= 0),
    // lq = {log S1, log S2, log V, log(U + S2)}
    double lg[4][CMAX], lq[4][CMAX];
    int m[CMAX];
    int alive_list[CMAX];
    int n_alive;
    double lref, lxref;
    double new_logZp[CMAX], new_logZp2[CMAX], new_logZXp[CMAX], new_logZpXp[CMAX], new_logXp[CMAX],
        new_logXp2[CMAX], dZ[CMAX], dZ2[CMAX], dZp2[CMAX], logw[CMAX];
};

// On this GPU one FP64 warp instruction occupies the SM sub-partition's FP64
// pipe for many cycles whatever the number of active lanes, so the update below
// keeps FP64 transcendentals few and spread over lanes: per-cluster logs are
// tabled once (one lane each), the five log-sums of every cluster run on
// separate lanes, and the kill passes carry only as many target clusters as
// there are (NB = 1, 2, 4 or 8).

// S1, S2, U, V of the nb target clusters tgt[0..nb) (NB >= nb) over the kills
// (see the comment above EvScratch); writes E->S1/S2/U/V of the targets.
template <int NB>
__device__ void evidence_kill_pass(int k, const double *kL, const int *kP, EvScratch *E, const int *tgt_list, int nb,
                                   double lref, bool have_l)
{
    const int tid = threadIdx.x;
    const int ch = (k + EV_THREADS - 1) / EV_THREADS;
    const int j0 = min(k, tid * ch), j1 = min(k, j0 + ch);
    double R[NB], Vl[NB], Ul[NB], S1l[NB], S2l[NB];
    int tgt[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        R[b] = Vl[b] = Ul[b] = S1l[b] = S2l[b] = 0.0;
        tgt[b] = (b < nb) ? tgt_list[b] : -1;
    }
    if (tid < EV_THREADS) {
        for (int j = j0; j < j1; ++j) {
            const int q = kP[j];
            const double l = (have_l && kL[j] == kL[j]) ? exp(kL[j] - lref) : 0.0;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (tgt[b] == q) {
                    Vl[b] += l * R[b];
                    Ul[b] += l * S1l[b];
                    S1l[b] += l;
                    S2l[b] += l * l;
                }
                R[b] += E->coef[b][q] * l;
            }
        }
    }
    // exclusive scans over threads of R and S1: warp shuffle scans, then the
    // warp totals in order (a fixed order: deterministic)
    const int lane = tid & 31, warp = tid >> 5;
    for (int pass = 0; pass < 2; ++pass) {
        double v[NB], x[NB];
#pragma unroll
        for (int bb = 0; bb < NB; ++bb) x[bb] = v[bb] = (pass == 0) ? R[bb] : S1l[bb];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int bb = 0; bb < NB; ++bb) {
                const double y = __shfl_up_sync(0xffffffffu, x[bb], o);
                if (lane >= o) x[bb] += y;
            }
        }
        if (lane == 31) {
#pragma unroll
            for (int bb = 0; bb < NB; ++bb) E->wtot[bb][warp] = x[bb];
        }
        __syncthreads();
#pragma unroll
        for (int bb = 0; bb < NB; ++bb) {
            double off = 0.0;
            for (int w2 = 0; w2 < warp; ++w2) off += E->wtot[bb][w2];
            const double excl = off + x[bb] - v[bb];
            if (pass == 0) Vl[bb] += S1l[bb] * excl;
            else Ul[bb] += S1l[bb] * excl;
        }
        __syncthreads();
    }
    // reductions over threads: warp trees, then the warp partials in order
    for (int qty = 0; qty < 4; ++qty) {
        double x[NB];
#pragma unroll
        for (int bb = 0; bb < NB; ++bb)
            x[bb] = qty == 0 ? S1l[bb] : (qty == 1 ? S2l[bb] : (qty == 2 ? Ul[bb] : Vl[bb]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int bb = 0; bb < NB; ++bb) x[bb] += __shfl_xor_sync(0xffffffffu, x[bb], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int bb = 0; bb < NB; ++bb) E->wtot[bb][warp] = x[bb];
        }
        __syncthreads();
        if (tid < nb) {
            double sacc = 0.0;
            for (int w2 = 0; w2 < EV_THREADS / 32; ++w2) sacc += E->wtot[tid][w2];
            const int c = tgt_list[tid];
            if (qty == 0) E->S1[c] = sacc;
            else if (qty == 1) E->S2[c] = sacc;
            else if (qty == 2) E->U[c] = sacc;
            else E->V[c] = sacc;
        }
        __syncthreads();
    }
}

// log(sum_i exp(t_i)) of the n terms term(0..n-1), by the largest term and one
// log; -inf when every term is -inf.
template <typename F>
__device__ __forceinline__ double log_sum(int n, F term)
{
    double m = -INFINITY;
    for (int i = 0; i < n; ++i) {
        const double t = term(i);
        m = (t > m) ? t : m;
    }
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += exp(term(i) - m);
    return m + log(s);
}

// kL[j] (FP64 log-likelihoods, ascending) and kP[j] (labels), j < k.  Updates
// st in place (the whole CTA calls it).  E->logw receives the log prior mass per
// kill of each cluster.  st->n and st->alive are updated.
__device__ void evidence_batch(Stats *st, double *logZ, double *logZ2, int k, const double *kL, const int *kP,
                               EvScratch *E)
{
    const int tid = threadIdx.x;
    if (tid < CMAX) {
        E->m[tid] = 0;
        E->S1[tid] = E->S2[tid] = E->U[tid] = E->V[tid] = 0.0;
    }
    if (tid == 0) {
        int na = 0;
        double lx = -INFINITY;
        for (int c = 0; c < CMAX; ++c)
            if (st->alive[c]) {
                E->alive_list[na++] = c;
                lx = fmax(lx, st->logXp[c]);
            }
        E->n_alive = na;
        // X_ref: largest cluster volume (keeps the coefficients a_{c,q} <= ~1)
        E->lxref = lx;
        // L_ref: largest finite log-likelihood of the batch
        double lr = -INFINITY;
        for (int j = k - 1; j >= 0; --j) {
            if (kL[j] == kL[j] && kL[j] > -INFINITY) {
                lr = kL[j];
                break;
            }
        }
        E->lref = lr;
    }
    __syncthreads();
    for (int j = tid; j < k; j += blockDim.x) atomicAdd(&E->m[kP[j]], 1);
    __syncthreads();
    const double lref = E->lref, lxref = E->lxref;
    const bool have_l = lref > -INFINITY && lref < INFINITY;
    const int nA = E->n_alive;
    // per-cluster count logs, one lane each
    for (int i = tid; i < 4 * nA; i += blockDim.x) {
        const int which = i / nA, c = E->alive_list[i - which * nA];
        const double n = (double)st->n[c], r = n - (double)E->m[c];
        double v;
        if (which == 0) v = log(n + 1.0);
        else if (which == 1) v = log(n + 2.0);
        else if (r <= 0.0) v = -INFINITY;
        else v = log(r + (which == 2 ? 1.0 : 2.0));
        E->lg[which][c] = v;
    }
    __syncthreads();
    for (int pb = 0; pb < nA; pb += EV_CB) {
        const int nb = min(EV_CB, nA - pb);
        // coefficient table a_{c,q} / X_ref for the target clusters c of this pass
        for (int i = tid; i < EV_CB * CMAX; i += blockDim.x) (&E->coef[0][0])[i] = 0.0;
        __syncthreads();
        for (int i = tid; i < nb * nA; i += blockDim.x) {
            const int b = i / nA, q = E->alive_list[i - b * nA], c = E->alive_list[pb + b];
            const double lc = (q == c) ? st->logXp2[c] - E->lg[1][c] - st->logXp[c]
                                       : st->logXX[q * CMAX + c] - E->lg[0][q] - st->logXp[c];
            E->coef[b][q] = exp(lc - lxref);
        }
        __syncthreads();
        const int *tl = E->alive_list + pb;
        if (nb <= 1) evidence_kill_pass<1>(k, kL, kP, E, tl, nb, lref, have_l);
        else if (nb <= 2) evidence_kill_pass<2>(k, kL, kP, E, tl, nb, lref, have_l);
        else if (nb <= 4) evidence_kill_pass<4>(k, kL, kP, E, tl, nb, lref, have_l);
        else evidence_kill_pass<8>(k, kL, kP, E, tl, nb, lref, have_l);
    }
    // logs of the batch sums, one lane each
    for (int i = tid; i < 4 * nA; i += blockDim.x) {
        const int which = i / nA, c = E->alive_list[i - which * nA];
        double v;
        if (which == 0) v = log(E->S1[c]);
        else if (which == 1) v = log(E->S2[c]);
        else if (which == 2) v = log(E->V[c]);
        else v = log(E->U[c] + E->S2[c]);
        E->lq[which][c] = v;
    }
    __syncthreads();
    // closed-form update of every live cluster (all right-hand sides old values):
    // five independent log-sums per cluster, one lane each
    const double LN2 = 0.69314718055994530942;
    const double L = lref;
    for (int i = tid; i < 5 * nA; i += blockDim.x) {
        const int which = i / nA, c = E->alive_list[i - which * nA];
        const int mc = E->m[c];
        const bool batch = mc > 0 && have_l;
        const double Xc = st->logXp[c], X2c = st->logXp2[c];
        const double ln1 = E->lg[0][c], ln2 = E->lg[1][c];
        const double lS1 = E->lq[0][c];
        if (which == 0) {
            // update3 summed: 2 e^L ZX_c S1/(n+1) + 2 e^2L X_c X_ref V/(n+1) + 2 e^2L X2_c S2/((n+1)(n+2))
            double dZ2 = -INFINITY;
            if (batch) {
                dZ2 = log_add(dZ2, LN2 + L + st->logZXp[c] + lS1 - ln1);
                dZ2 = log_add(dZ2, LN2 + 2.0 * L + Xc + lxref + E->lq[2][c] - ln1);
                dZ2 = log_add(dZ2, LN2 + 2.0 * L + X2c + E->lq[1][c] - ln1 - ln2);
            }
            E->dZ2[c] = dZ2;
        } else if (which == 1) {
            // update4 summed: 2 e^L Z_cX_c S1/(n+1) + 2 e^2L X2_c (U + S2)/((n+1)(n+2))
            double dZp2 = -INFINITY;
            if (batch) {
                dZp2 = log_add(dZp2, LN2 + L + st->logZpXp[c] + lS1 - ln1);
                dZp2 = log_add(dZp2, LN2 + 2.0 * L + X2c + E->lq[3][c] - ln1 - ln2);
            }
            E->dZp2[c] = dZp2;
        } else if (which == 2) {
            // update5/6: ZX_c -> rho (ZX_c + e^L [X2_c S1_c/(n_c+2) + sum_{q != c} XX_qc S1_q/(n_q+1)])
            double inner = st->logZXp[c];
            if (have_l) {
                // terms: ZX_c, the cluster's own kills, then the other clusters with kills (ascending q)
                const int a = i - which * nA;  // c's place in the alive list
                inner = log_sum(nA + 1, [&](int t) -> double {
                    if (t == 0) return st->logZXp[c];
                    if (t == 1) return mc > 0 ? L + X2c + lS1 - ln2 : -INFINITY;
                    const int q = E->alive_list[(t - 2 < a) ? t - 2 : t - 1];
                    return E->m[q] > 0 ? L + st->logXX[q * CMAX + c] + E->lq[0][q] - E->lg[0][q] : -INFINITY;
                });
            }
            const double lrho = E->lg[2][c] - ln1;
            E->new_logZXp[c] = (E->lg[2][c] > -INFINITY) ? inner + lrho : -INFINITY;
        } else if (which == 3) {
            // update7: Z_cX_c -> rho (Z_cX_c + e^L X2_c S1_c/(n_c+2))
            double inner2 = st->logZpXp[c];
            if (batch) inner2 = log_add(inner2, L + X2c + lS1 - ln2);
            const double lrho = E->lg[2][c] - ln1;
            E->new_logZpXp[c] = (E->lg[2][c] > -INFINITY) ? inner2 + lrho : -INFINITY;
        } else {
            // update0/1 summed: dZ_c = X_c S1_c e^L / (n_c + 1)
            const double dZ = batch ? Xc - ln1 + lS1 + L : -INFINITY;
            E->dZ[c] = dZ;
            E->new_logZp[c] = log_add(st->logZp[c], dZ);
            E->logw[c] = Xc - ln1;
            const bool left = E->lg[2][c] > -INFINITY;  // points of c survive the batch
            const double lrho = left ? E->lg[2][c] - ln1 : -INFINITY;
            E->new_logXp[c] = Xc + lrho;
            E->new_logXp2[c] = left ? X2c + E->lg[2][c] + E->lg[3][c] - ln1 - ln2 : -INFINITY;
        }
    }
    __syncthreads();
    // second level: Z_c^2 of every cluster, log Z and log Z^2 of the run (one lane each)
    for (int i = tid; i < nA + 2; i += blockDim.x) {
        if (i < nA) {
            const int c = E->alive_list[i];
            E->new_logZp2[c] = log_add(st->logZp2[c], E->dZp2[c]);
        } else {
            const double *d = (i == nA) ? E->dZ : E->dZ2;
            double *out = (i == nA) ? logZ : logZ2;
            const double z0 = *out;
            *out = log_sum(nA + 1, [&](int t) -> double { return t == 0 ? z0 : d[E->alive_list[t - 1]]; });
        }
    }
    // update9 for the cross moments (old counts), then commit
    for (int i = tid; i < CMAX * CMAX; i += blockDim.x) {
        const int c = i / CMAX, q = i % CMAX;
        if (c == q || !st->alive[c] || !st->alive[q]) continue;
        if (E->lg[2][c] == -INFINITY || E->lg[2][q] == -INFINITY) st->logXX[i] = -INFINITY;
        else st->logXX[i] += E->lg[2][c] - E->lg[0][c] + E->lg[2][q] - E->lg[0][q];
    }
    __syncthreads();
    if (tid < CMAX && st->alive[tid]) {
        const int c = tid;
        st->logZp[c] = E->new_logZp[c];
        st->logZp2[c] = E->new_logZp2[c];
        st->logZXp[c] = E->new_logZXp[c];
        st->logZpXp[c] = E->new_logZpXp[c];
        st->logXp[c] = E->new_logXp[c];
        st->logXp2[c] = E->new_logXp2[c];
        st->n[c] -= E->m[c];
        if (st->n[c] <= 0) {
            // Algorithm 3: a cluster without points is removed
            st->alive[c] = 0;
            st->n[c] = 0;
            st->logZp[c] = st->logZp2[c] = st->logZXp[c] = st->logZpXp[c] = -INFINITY;
            st->logXp[c] = st->logXp2[c] = -INFINITY;
        }
    }
    __syncthreads();
    for (int i = tid; i < CMAX * CMAX; i += blockDim.x) {
        const int c = i / CMAX, q = i % CMAX;
        if (!st->alive[c] || !st->alive[q]) st->logXX[i] = -INFINITY;
    }
    __syncthreads();
}

// ------------------------------------------------------------------------
// Final sweep of a terminated run (Algorithm 3, last loop): every live point is
// killed in ascending (log L, slot) order and enters the statistics and the dead
// records.  One CTA per run.  dynamic smem: npow2 keys (8 B) | EvScratch | Stats
// ------------------------------------------------------------------------
constexpr int SEL_THREADS = 256;

__device__ void final_sweep_body(DevCtx C, int r)
{
    extern __shared__ unsigned char sraw[];
    const RunDesc &D = C.desc[r];
    RunState *S = C.state + r;
    const int n = D.n_live;
    const int npow = next_pow2(n);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(sraw);
    EvScratch *E = reinterpret_cast<EvScratch *>(sraw + key_region_bytes(n));
    // the run's statistics live in shared memory for the whole kernel
    Stats *st = reinterpret_cast<Stats *>(sraw + key_region_bytes(n) + ((sizeof(EvScratch) + 15) & ~size_t(15)));
    {
        const int4 *src = reinterpret_cast<const int4 *>(C.stats + r);
        int4 *dst = reinterpret_cast<int4 *>(st);
        for (int i = threadIdx.x; i < (int)(sizeof(Stats) / 16); i += blockDim.x) dst[i] = src[i];
    }
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const float *logl = C.logl + D.pt_off;
    const int k = n;  // every live point is killed

    // ---- ascending (log L, slot) order; NaN first
    for (int i = tid; i < npow; i += blockDim.x)
        keys[i] = (i < n) ? ((unsigned long long)float_key(logl[i]) << 32) | (unsigned)i : ~0ull;
    __syncthreads();
    block_bitonic_sort(keys, npow);
    for (int i = tid; i < n; i += blockDim.x) C.order[D.pt_off + i] = (int)(keys[i] & 0xffffffffu);
    if (tid == 0) {
        s_abort = 0;
        if (S->n_dead + k > D.dead_cap) {
            S->status = NS_ERR_CAPACITY;
            S->done = 1;
            S->final_done = 1;
            s_abort = 1;
        }
    }
    __syncthreads();
    if (s_abort) return;
    // ---- kill list in the key buffer: kL (double[k]) then kP (int[k])
    double *kL = reinterpret_cast<double *>(keys);
    int *kP = reinterpret_cast<int *>(kL + k);
    int *ordr = C.order + D.pt_off;
    // (keys are dead after `order` is written; read slots back from global)
    __syncthreads();
    for (int j = tid; j < k; j += blockDim.x) {
        const int s = ordr[j];
        kL[j] = (double)logl[s];
        kP[j] = C.label[D.pt_off + s];
    }
    __syncthreads();
    const long dbase = D.dead_off + S->n_dead;
    evidence_batch(st, &S->logz, &S->logz2, k, kL, kP, E);
    auto store_stats = [&]() {
        __syncthreads();
        const int4 *src = reinterpret_cast<const int4 *>(st);
        int4 *dst = reinterpret_cast<int4 *>(C.stats + r);
        for (int i = threadIdx.x; i < (int)(sizeof(Stats) / 16); i += blockDim.x) dst[i] = src[i];
    };
    // dead records: log L, log prior mass, label, x
    for (int j = tid; j < k; j += blockDim.x) {
        if (!gg_in(dbase + j - D.dead_off, D.dead_cap, S)) continue;
        D.dead_logl[dbase + j] = (float)kL[j];
        D.dead_logw[dbase + j] = E->logw[kP[j]];
        D.dead_label[dbase + j] = kP[j];
        // the final sweep has no walkers: archive x here
        const int s = ordr[j];
        const float *src = C.fa + D.x_off + (long)s * D.d_pad;
        float *dst = D.dead_x + (dbase + j) * D.d_pad;
        for (int e = 0; e < D.d_pad; ++e) dst[e] = src[e];
    }
    __syncthreads();
    if (tid == 0) {
        S->n_dead += k;
        S->final_done = 1;
        if (!(S->logz == S->logz)) S->status = NS_ERR_NUMERIC;
    }
    store_stats();
}

// ------------------------------------------------------------------------
// Selection and spawn of one iteration (Algorithm 3), one CTA of SORT_THREADS
// per run.  Only the prior volumes enter the spawn, and their batch update is a
// closed form (X_c (n_c - m_c + 1)/(n_c + 1)), so the FP64 moment update of
// Appendix H (k_evidence) runs beside the HSS phases instead of before them.
// dynamic smem: key region (npow2 x 8 bytes, reused for the survivor lists).
// ------------------------------------------------------------------------
constexpr int SORT_THREADS = 1024;

__device__ void sort_body(DevCtx C, int r, unsigned char *sraw)
{
    const RunDesc &D = C.desc[r];
    RunState *S = C.state + r;
    if (S->done) return;
    const Stats *st = C.stats + r;
    const int n = D.n_live, k = D.k;
    const int npow = next_pow2(n);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(sraw);
    __shared__ int s_abort, s_na, s_alive_list[CMAX];
    __shared__ int s_m[CMAX], s_cnt[CMAX], s_start[CMAX], s_surv[CMAX];
    __shared__ double s_w[CMAX], s_cum[CMAX], s_total;
    __shared__ int s_wsum[SORT_THREADS / 32];
    const float *logl = C.logl + D.pt_off;
    const int *label = C.label + D.pt_off;
    int *ordr = C.order + D.pt_off;

    // ---- ascending (log L, slot) order; NaN first
    for (int i = tid; i < npow; i += blockDim.x)
        keys[i] = (i < n) ? ((unsigned long long)float_key(logl[i]) << 32) | (unsigned)i : ~0ull;
    if (tid < CMAX) {
        s_m[tid] = 0;
        s_cnt[tid] = 0;
    }
    __syncthreads();
    block_bitonic_sort(keys, npow);
    for (int i = tid; i < n; i += blockDim.x) ordr[i] = (int)(keys[i] & 0xffffffffu);
    if (tid == 0) {
        s_abort = 0;
        if (S->n_dead + k > D.dead_cap) {
            S->status = NS_ERR_CAPACITY;
            S->done = 1;
            S->final_done = 1;
            s_abort = 1;
        }
    }
    __syncthreads();
    if (s_abort) return;
    // ---- dead records of the kills (log L, label); x rows are archived by the walkers
    const long dbase = S->n_dead;
    for (int j = tid; j < k; j += blockDim.x) {
        const int s0 = (int)(keys[j] & 0xffffffffu);
        const int c = label[s0];
        if (gg_in(dbase + j, D.dead_cap, S) && gg_in(s0, D.n_live, S)) {
            D.dead_logl[dbase + j] = logl[s0];
            D.dead_label[dbase + j] = c;
        }
        atomicAdd(&s_m[c], 1);
    }
    __syncthreads();
    // ---- prior volumes after the kills, in closed form; spawn weights Xbar_c / max Xbar
    if (tid < CMAX) {
        const int c = tid;
        const int left = st->alive[c] ? st->n[c] - s_m[c] : 0;
        s_surv[c] = left > 0 ? left : 0;
        s_w[c] = (left > 0) ? st->logXp[c] + log((double)left + 1.0) - log((double)st->n[c] + 1.0) : -INFINITY;
    }
    __syncthreads();
    if (tid == 0) {
        double mx = -INFINITY;
        int na = 0, off = 0;
        for (int c = 0; c < CMAX; ++c) {
            s_start[c] = off;
            if (s_surv[c] > 0) {
                mx = fmax(mx, s_w[c]);
                s_alive_list[na++] = c;
                off += s_surv[c];
            }
        }
        s_na = na;
        s_total = mx;
    }
    __syncthreads();
    if (tid < CMAX) s_w[tid] = (s_surv[tid] > 0) ? exp(s_w[tid] - s_total) : 0.0;
    __syncthreads();
    if (tid == 0) {
        // cumulative weights in cluster-id order (FP64)
        double cum = 0.0;
        for (int a = 0; a < s_na; ++a) {
            const int c = s_alive_list[a];
            cum += s_w[c];
            s_cum[c] = cum;
        }
        s_total = cum;
        if (s_na == 0) {
            S->status = NS_ERR_NUMERIC;
            S->done = 1;
        }
    }
    __syncthreads();
    if (S->done) return;
    // ---- survivors of each cluster in slot order: ordered compaction, one cluster at a time
    unsigned char *killed = reinterpret_cast<unsigned char *>(keys);  // keys are no longer needed
    int *surv = reinterpret_cast<int *>(sraw + ((npow + 15) & ~15));
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) killed[i] = 0;
    __syncthreads();
    for (int j = tid; j < k; j += blockDim.x) killed[ordr[j]] = 1;
    __syncthreads();
    const int na = s_na;
    for (int a = 0; a < na; ++a) {
        const int c = s_alive_list[a];
        int base = s_start[c];
        for (int i0 = 0; i0 < n; i0 += blockDim.x) {
            const int i = i0 + tid;
            const int f = (i < n && !killed[i] && label[i] == c) ? 1 : 0;
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (lane == 0) s_wsum[warp] = __popc(bal);
            __syncthreads();
            int off = base;
            for (int w2 = 0; w2 < warp; ++w2) off += s_wsum[w2];
            if (f) {
                const int pos = off + __popc(bal & ((1u << lane) - 1u));
                if (pos < n) surv[pos] = i;
            }
            int tot = 0;
            for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) tot += s_wsum[w2];
            __syncthreads();
            base += tot;
        }
        if (tid == 0 && base - s_start[c] != s_surv[c]) s_abort = 1;  // counts and labels disagree
    }
    __syncthreads();
    if (s_abort) {
        if (tid == 0) {
            S->status = NS_ERR_NUMERIC;
            S->done = 1;
        }
        return;
    }
    // ---- spawn: cluster with probability Xbar_c / sum Xbar, then a uniform surviving member
    const uint32_t iter = (uint32_t)S->iter;
    for (int j = tid; j < k; j += blockDim.x) {
        const U4 w = rng_block(D, iter, P_CLUSTER, j, 0, 0);
        const double target = u01_52(w.x, w.y) * s_total;
        int chosen = s_alive_list[na - 1];
        for (int a = 0; a < na; ++a) {
            const int c = s_alive_list[a];
            if (target < s_cum[c]) {
                chosen = c;
                break;
            }
        }
        const int m = s_surv[chosen];
        const U4 w2 = rng_block(D, iter, P_START, j, 0, 0);
        const int pick = (int)(((unsigned long long)w2.x * (unsigned long long)m) >> 32);
        C.start_slot[D.w_off + j] = surv[s_start[chosen] + pick];
        C.new_label[D.w_off + j] = chosen;
        atomicAdd(&s_cnt[chosen], 1);
    }
    __syncthreads();
    if (tid < CMAX) {
        S->kill_cnt[tid] = s_m[tid];
        S->spawn_cnt[tid] = s_cnt[tid];
    }
    if (tid == 0) {
        S->lstar = (double)logl[ordr[k - 1]];
        if (!(S->lstar == S->lstar)) {
            // more than half the live points have a NaN log-likelihood: no slice to sample
            S->status = NS_ERR_NUMERIC;
            S->done = 1;
        }
        S->dead_base = dbase;
        S->n_dead = dbase + k;
        S->ev_pending = 1;
        S->wcount[0] = S->wcount[1] = S->wcount[2] = 0;
        S->t_save = 0;
        S->t_stop = 0;
        S->n_in = 0;
        S->n_out = 0;
        S->n_fold = 0;
        S->wcount1 = 0;
        S->t_save1 = 0;
        S->t_stop1 = 0;
        S->remain_min = k;
        S->remain_max = k;
        S->rec_overflow = 0;
    }
}

// ------------------------------------------------------------------------
// Appendix H statistics of the iteration's kills (FP64), beside the HSS phases.
// Reads the kills from the dead records, writes their log prior masses, applies
// the spawn counts and the XL statistic.  dynamic smem: kill arrays | EvScratch | Stats
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(SEL_THREADS) k_evidence(DevCtx C, int r0)
{
    extern __shared__ unsigned char sraw[];
    const int r = r0 + blockIdx.x;
    const RunDesc &D = C.desc[r];
    RunState *S = C.state + r;
    if (!S->ev_pending) return;
    const int k = D.k;
    double *kL = reinterpret_cast<double *>(sraw);
    int *kP = reinterpret_cast<int *>(kL + k);
    EvScratch *E = reinterpret_cast<EvScratch *>(sraw + key_region_bytes(D.n_live));
    Stats *st = reinterpret_cast<Stats *>(sraw + key_region_bytes(D.n_live) + ((sizeof(EvScratch) + 15) & ~size_t(15)));
    const int tid = threadIdx.x;
    {
        const int4 *src = reinterpret_cast<const int4 *>(C.stats + r);
        int4 *dst = reinterpret_cast<int4 *>(st);
        for (int i = tid; i < (int)(sizeof(Stats) / 16); i += blockDim.x) dst[i] = src[i];
    }
    const long dbase = S->dead_base;
    for (int j = tid; j < k; j += blockDim.x) {
        const bool in = gg_in(dbase + j, D.dead_cap, S);
        kL[j] = in ? (double)D.dead_logl[dbase + j] : 0.0;
        kP[j] = in ? D.dead_label[dbase + j] : 0;
    }
    __syncthreads();
    evidence_batch(st, &S->logz, &S->logz2, k, kL, kP, E);
    for (int j = tid; j < k; j += blockDim.x)
        if (gg_in(dbase + j, D.dead_cap, S)) D.dead_logw[dbase + j] = E->logw[kP[j]];
    __syncthreads();
    if (tid < CMAX && st->alive[tid]) st->n[tid] += S->spawn_cnt[tid];
    __syncthreads();
    if (tid < 32) {
        // XL statistic on the dead-point sequence: log X (after the kills) + L*, as
        // one log-sum over the live clusters (their exponentials one lane each)
        double m = -INFINITY;
        int na = 0;
        for (int c = tid; c < CMAX; c += 32)
            if (st->alive[c]) {
                m = fmax(m, st->logXp[c]);
                ++na;
            }
        for (int o = 16; o > 0; o >>= 1) {
            m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            na += __shfl_xor_sync(0xffffffffu, na, o);
        }
        double e = 0.0;
        if (m > -INFINITY)
            for (int c = tid; c < CMAX; c += 32)
                if (st->alive[c]) e += exp(st->logXp[c] - m);
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (tid == 0) {
            S->log_xl = ((m > -INFINITY) ? m + log(e) : -INFINITY) + S->lstar;
            S->n_clusters = na;
            S->ev_pending = 0;
        }
    }
    {
        const int4 *src = reinterpret_cast<const int4 *>(st);
        int4 *dst = reinterpret_cast<int4 *>(C.stats + r);
        for (int i = tid; i < (int)(sizeof(Stats) / 16); i += blockDim.x) dst[i] = src[i];
    }
}

__global__ void __launch_bounds__(SEL_THREADS) k_final(DevCtx C, int r0)
{
    const int r = r0 + blockIdx.x;
    if (!C.state[r].done || C.state[r].final_done) return;
    final_sweep_body(C, r);
}

size_t sort_smem_bytes(int n_live_max)
{
    const size_t np = (size_t)next_pow2(n_live_max);
    const size_t a = np * 8, b = ((np + 15) & ~size_t(15)) + 4 * (size_t)n_live_max;
    return a > b ? a : b;
}

size_t select_smem_bytes(int n_live_max)
{
    return key_region_bytes(n_live_max) + ((sizeof(EvScratch) + 15) & ~size_t(15)) + sizeof(Stats);
}

// ------------------------------------------------------------------------
// Iteration tail: step-size rule (Algorithm 3), counters, termination test.
// ------------------------------------------------------------------------
__global__ void k_tail(DevCtx C, int r0)
{
    const int r = r0 + blockIdx.x;
    const RunDesc &D = C.desc[r];
    RunState *S = C.state + r;
    if (S->done) return;
    __shared__ float s_max[32];
    // L_max over the live points (classic termination)
    float m = -INFINITY;
    for (int i = threadIdx.x; i < D.n_live; i += blockDim.x) {
        const float v = C.logl[D.pt_off + i];
        if (v > m) m = v;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_max[w]);
    // the reflections per step (with box_fold and fold_counts, the box's exact reflections count)
    const long tot = S->n_in + S->n_out;
    const long nrefl = S->n_out + ((D.box_fold && D.fold_counts) ? S->n_fold : 0);
    const double out_frac = tot > 0 ? (double)nrefl / (double)tot : 0.0;
    if (out_frac > D.out_hi) S->dt *= 0.9;
    else if (out_frac < D.out_lo) S->dt *= 1.1;
    S->n_like += (long)D.k * S->t_stop;
    S->n_steps_total += (long)D.k * S->t_stop;
    S->n_rec_overflow += S->rec_overflow;
    S->lmax_live = m;
    S->iter += 1;
    S->term_pending = 1;
}

// Termination test of the last finished iteration (Algorithm 3): runs once its
// FP64 statistics are in, which lets them overlap the tail and the next
// iteration's k-NN.  XL peak on the dead-point sequence (termination 0) or
// X L_max < tol Z (termination 1); then the iteration cap.
__device__ void term_body(DevCtx C, int r)
{
    const RunDesc &D = C.desc[r];
    RunState *S = C.state + r;
    if (S->done || !S->term_pending) return;
    S->term_pending = 0;
    if (S->log_xl > S->log_xl_max) S->log_xl_max = S->log_xl;
    bool stop;
    if (D.termination == 0) {
        stop = (S->log_xl - S->log_xl_max) < D.log_tol;
    } else {
        double lx = -INFINITY;
        const Stats *st = C.stats + r;
        for (int c = 0; c < CMAX; ++c)
            if (st->alive[c]) lx = log_add(lx, st->logXp[c]);
        stop = (lx + (double)S->lmax_live) < D.log_tol + S->logz;
    }
    if (S->n_clusters > S->max_clusters) S->max_clusters = S->n_clusters;
    if (stop) {
        S->terminated = 1;
        S->done = 1;
    } else if (S->iter >= D.max_iters) {
        S->status = NS_ERR_NOT_DONE;
        S->done = 1;
    }
}

__global__ void k_term(DevCtx C, int r0, int n_runs)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_runs) term_body(C, r0 + t);
}

// Reservoir replay over the recorded window and emission of every walker's new
// point, one warp per walker: lane l reads the records of steps 32 m + l + 1, the
// saved steps of a round are counted with a ballot, and the last step whose
// acceptance test passes (word * count < 2^32, count = rank among the saved
// steps) is the pick -- the same sequence of decisions as the sequential reservoir.
constexpr int PICK_WARPS = 4;

__global__ void __launch_bounds__(PICK_WARPS * 32) k_hss_pick(DevCtx C, const int *run_list, RecView R,
                                                              const long *rec_base)
{
    const int r = run_list[blockIdx.y];
    const RunDesc &D = C.desc[r];
    RunState *S = C.state + r;
    if (S->done || S->rec_overflow) return;
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * PICK_WARPS + (threadIdx.x >> 5);
    const int W = D.k, dp = D.d_pad;
    const int ts0 = max(S->t_save1, 1), tstop = S->t_stop1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the tail and the counters read the window of the three-phase form
        S->t_save = S->t_save1;
        S->t_stop = S->t_stop1;
        S->t_stop_last = S->t_stop1;
    }
    if (w >= W) return;
    const long base = rec_base[r] + (long)w * R.rec_len;
    // the window lies inside this walker's record rows
    if (tstop > 0 && !gg_in(tstop - 1, R.rec_len, S)) return;
    // the steps of the window that enter the reservoir: inside steps from t_save on;
    // with pick_all every step, a drawn outside step rejecting (the start point)
    int pick = 0, count = 0, nout = 0, nfold = 0;
    bool pick_out = false;
    for (int t0 = 1; t0 <= tstop; t0 += 32) {
        const int t = t0 + lane;
        uint2 m = make_uint2(0u, 0u);
        if (t <= tstop) m = R.meta[base + t - 1];
        const bool in_win = t <= tstop;
        const bool outside = in_win && (m.y & 1u) != 0u;
        const bool saved = in_win && (!outside || D.pick_all || D.midpoint) && t >= ts0;
        const unsigned smask = __ballot_sync(0xffffffffu, saved);
        const int cnt = count + __popc(smask & ((1u << lane) - 1u)) + 1;
        const bool acc = saved && (D.keep_last || ((static_cast<uint64_t>(m.x) * static_cast<uint64_t>(cnt)) >> 32) == 0);
        const unsigned amask = __ballot_sync(0xffffffffu, acc);
        const unsigned omask = __ballot_sync(0xffffffffu, outside);
        const unsigned fmask = __ballot_sync(0xffffffffu, in_win && (m.y & 2u) != 0u);
        if (amask) {
            const int hl = 31 - __clz(amask);
            pick = t0 + hl;
            pick_out = (omask >> hl) & 1u;
        }
        count += __popc(smask);
        nout += __popc(omask);
        nfold += __popc(fmask);
    }
    // rejected: the walker keeps its start point (with midpoint the drawn state is tested
    // against L* by k_eval_new: the outside flag is that of the half step)
    if (pick_out && !D.midpoint) pick = 0;
    const int slot = C.order[D.pt_off + w];
    if (!gg_in(slot, D.n_live, S) || !gg_in(C.start_slot[D.w_off + w], D.n_live, S)) return;
    float *dst = C.fa + D.x_off + (long)slot * dp;
    const float *src = (pick > 0) ? R.x + (base + pick - 1) * R.xs
                                  : C.fa + D.x_off + (long)C.start_slot[D.w_off + w] * dp;
    for (int c = lane; c < dp; c += 32) dst[c] = src[c];
    if (lane == 0) {
        C.logl[D.pt_off + slot] = (pick > 0) ? R.ll[base + pick - 1] : C.logl[D.pt_off + C.start_slot[D.w_off + w]];
        if (D.midpoint) C.wint[(D.w_off + w) * WINT + 10] = (pick > 0) ? 1 : 0;
        C.label[D.pt_off + slot] = C.new_label[D.w_off + w];
        atomicAdd(reinterpret_cast<unsigned long long *>(&S->n_in), static_cast<unsigned long long>(tstop - nout));
        atomicAdd(reinterpret_cast<unsigned long long *>(&S->n_out), static_cast<unsigned long long>(nout));
        if (nfold) atomicAdd(reinterpret_cast<unsigned long long *>(&S->n_fold), static_cast<unsigned long long>(nfold));
        if (pick <= 0) C.wint[(D.w_off + w) * WINT + 6] = 1;
    }
}

// ------------------------------------------------------------------------
// Cluster regions of the new points (the bookkeeping of Appendix H holds when
// the live points of a cluster lie in that cluster's region only)
// ------------------------------------------------------------------------
// Nearest-survivor search, one query per lane: a CTA of TER_WARPS warps serves 32
// queries (new points) held transposed in shared memory (q[c * 33 + lane], no bank
// conflicts).  The candidate rows come through shared memory in tiles of TER_TILE
// rows (rows padded with zeros to ds = d rounded up to 4); warp w stages and scans
// rows w, w + TER_WARPS, ... of a tile (TER_TILE / TER_WARPS rows, their loads in
// flight together, one accumulator each; only warp barriers) and walks the
// coordinates four at a time: the query's four from shared memory once, each row's
// four as one broadcast float4.  Squared
// distances accumulate over the coordinates in order (FP32, round to nearest; the
// zero padding adds fma(0, 0, s) = s), the order the oracle uses; ties go to the lower
// candidate key, so the result does not depend on the scan order.  Returns, in every
// lane of warp 0, the key of its query's nearest candidate (-1 if none).
constexpr int TER_WARPS = 4;
constexpr int TER_TILE = 32;
constexpr int TER_ROWS = TER_TILE / TER_WARPS;  // rows of a tile per warp

__device__ __forceinline__ void ter_take(float s, int k, float &best, int &bk)
{
    if (s < best || (s == best && k < bk)) {
        best = s;
        bk = k;
    }
}

__host__ __device__ inline int ter_ds(int d) { return (d + 3) & ~3; }

template <typename RowF, typename KeyF>
__device__ __forceinline__ int tile_nearest(const float *q, int d, int m, RowF cand, KeyF key, float *mb, int *mk,
                                            float *ct)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ds = ter_ds(d);
    float best = INFINITY;
    int bk = 0x7fffffff;
    for (int t0 = 0; t0 < m; t0 += TER_TILE) {
        const int nt = min(TER_TILE, m - t0);
        // each warp stages its own rows of the tile (rows warp + TER_WARPS j): the row
        // addresses first, then every row's loads in flight together, coalesced over lanes
        const float *rp[TER_ROWS];
#pragma unroll
        for (int j = 0; j < TER_ROWS; ++j) {
            const int r = warp + TER_WARPS * j;
            rp[j] = (r < nt) ? cand(t0 + r) : nullptr;
        }
        __syncwarp();  // this warp's previous rows are consumed
        for (int c = lane; c < ds; c += 32) {
            float v[TER_ROWS];
#pragma unroll
            for (int j = 0; j < TER_ROWS; ++j) v[j] = (rp[j] != nullptr && c < d) ? __ldg(rp[j] + c) : 0.f;
#pragma unroll
            for (int j = 0; j < TER_ROWS; ++j) ct[(warp + TER_WARPS * j) * ds + c] = v[j];
        }
        __syncwarp();
        float acc[TER_ROWS];
#pragma unroll
        for (int j = 0; j < TER_ROWS; ++j) acc[j] = 0.f;
        for (int c0 = 0; c0 < ds; c0 += 4) {
            const float q0 = q[c0 * 33 + lane], q1 = q[(c0 + 1) * 33 + lane];
            const float q2 = q[(c0 + 2) * 33 + lane], q3 = q[(c0 + 3) * 33 + lane];
#pragma unroll
            for (int j = 0; j < TER_ROWS; ++j) {
                const int r = warp + TER_WARPS * j;
                if (r < nt) {
                    const float4 v = *reinterpret_cast<const float4 *>(ct + r * ds + c0);
                    float df = q0 - v.x;
                    acc[j] = __fmaf_rn(df, df, acc[j]);
                    df = q1 - v.y;
                    acc[j] = __fmaf_rn(df, df, acc[j]);
                    df = q2 - v.z;
                    acc[j] = __fmaf_rn(df, df, acc[j]);
                    df = q3 - v.w;
                    acc[j] = __fmaf_rn(df, df, acc[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < TER_ROWS; ++j) {
            const int r = warp + TER_WARPS * j;
            if (r < nt) ter_take(acc[j], key(t0 + r), best, bk);
        }
    }
    mb[warp * 32 + lane] = best;
    mk[warp * 32 + lane] = bk;
    __syncthreads();
    if (warp == 0) {
        for (int w = 1; w < TER_WARPS; ++w) ter_take(mb[w * 32 + lane], mk[w * 32 + lane], best, bk);
    }
    return bk == 0x7fffffff ? -1 : bk;
}

// Shared memory of the territory kernels: the query tile, the candidate tile and the
// warps' partial minima (the query and candidate tiles padded to ds coordinates).
__host__ __device__ inline size_t territory_smem_bytes(int d)
{
    return sizeof(float) * (size_t)ter_ds(d) * (33 + TER_TILE) + (sizeof(float) + sizeof(int)) * TER_WARPS * 32;
}

// Walker w's new point (slot order[w]) stays only if its nearest surviving point
// (slots order[k .. n_live), ties to the lower slot) carries the label it was
// spawned with; otherwise the slot takes the walker's start point and its log L.
// Runs with clustering and the region rule on; skipped while every survivor has
// one label (the spawned label is always a survivor's).
__global__ void __launch_bounds__(TER_WARPS * 32) k_territory(DevCtx C, int r0)
{
    extern __shared__ float tsm[];
    __shared__ int s_mixed;
    const int r = r0 + blockIdx.y;
    const RunDesc &D = C.desc[r];
    const RunState *S = C.state + r;
    if (S->done || !D.clustering || !D.territory) return;
    const int n = D.n_live, k = D.k, dp = D.d_pad, d = D.d;
    const int w0 = blockIdx.x * 32;
    if (w0 >= k) return;
    const int *ord = C.order + D.pt_off;
    const int *lab = C.label + D.pt_off;
    if (threadIdx.x == 0) s_mixed = 0;
    __syncthreads();
    const int l0 = lab[ord[k]];
    bool mixed = false;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) mixed |= (lab[ord[i]] != l0);
    if (mixed) s_mixed = 1;
    __syncthreads();
    if (!s_mixed) return;
    const float *xs = C.fa + D.x_off;
    const int ds = ter_ds(d);
    float *q = tsm;
    float *ct = tsm + (size_t)ds * 33;
    float *mb = ct + (size_t)ds * TER_TILE;
    int *mk = reinterpret_cast<int *>(mb + TER_WARPS * 32);
    {
        // warp w fills queries w, w + TER_WARPS, ...: the rows' addresses first, then the
        // rows' loads in flight together, coalesced over the lanes
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const float *qp[TER_ROWS];
#pragma unroll
        for (int i = 0; i < TER_ROWS; ++i) {
            const int j = warp + TER_WARPS * i;
            qp[i] = (w0 + j < k) ? xs + (long)ord[w0 + j] * dp : nullptr;
        }
        for (int c = lane; c < ds; c += 32) {
            float v[TER_ROWS];
#pragma unroll
            for (int i = 0; i < TER_ROWS; ++i) v[i] = (qp[i] != nullptr && c < d) ? qp[i][c] : 0.f;
#pragma unroll
            for (int i = 0; i < TER_ROWS; ++i) q[c * 33 + warp + TER_WARPS * i] = v[i];
        }
    }
    __syncthreads();
    const int near = tile_nearest(q, d, n - k, [&](int i) { return xs + (long)ord[k + i] * dp; },
                                  [&](int i) { return ord[k + i]; }, mb, mk, ct);
    const int lane = threadIdx.x & 31, w = w0 + lane;
    const bool reject = (threadIdx.x < 32) && w < k && near >= 0 && lab[near] != C.new_label[D.w_off + w];
    // the warps copy the rejected walkers' start points (warp w: walkers w, w + TER_WARPS, ...)
    __shared__ int s_rej[32];
    if (threadIdx.x < 32) s_rej[lane] = reject ? 1 : 0;
    __syncthreads();
    for (int j = threadIdx.x >> 5; j < 32; j += TER_WARPS) {
        if (!s_rej[j]) continue;
        const int ww = w0 + j;
        const int slot = ord[ww], s0 = C.start_slot[D.w_off + ww];
        for (int c = lane; c < dp; c += 32) C.fa[D.x_off + (long)slot * dp + c] = xs[(long)s0 * dp + c];
        if (lane == 0) C.logl[D.pt_off + slot] = C.logl[D.pt_off + s0];
    }
}

// Component form for the tests: keep[j] = 1 if the nearest of the m_s survivor
// rows surv[m_s][d] (ties to the lower row) to xn[j] carries label want[j].
__global__ void __launch_bounds__(TER_WARPS * 32) k_territory_plain(const float *surv, const int *surv_label, int m_s,
                                                                    const float *xn, const int *want, int k, int d,
                                                                    int *keep)
{
    extern __shared__ float tsm[];
    const int w0 = blockIdx.x * 32;
    const int ds = ter_ds(d);
    float *q = tsm;
    float *ct = tsm + (size_t)ds * 33;
    float *mb = ct + (size_t)ds * TER_TILE;
    int *mk = reinterpret_cast<int *>(mb + TER_WARPS * 32);
    for (int e = threadIdx.x; e < 32 * ds; e += blockDim.x) {
        const int j = e / ds, c = e - j * ds;
        q[c * 33 + j] = (w0 + j < k && c < d) ? xn[(long)(w0 + j) * d + c] : 0.f;
    }
    __syncthreads();
    const int near =
        tile_nearest(q, d, m_s, [&](int i) { return surv + (long)i * d; }, [&](int i) { return i; }, mb, mk, ct);
    const int j = w0 + threadIdx.x;
    if (threadIdx.x < 32 && j < k) keep[j] = (near < 0 || surv_label[near] == want[j]) ? 1 : 0;
}

// ------------------------------------------------------------------------
// Cluster finding (Algorithm 4)
// ------------------------------------------------------------------------
// k-NN ranks 1..KNN_K of point i among the points with the same label, by
// ascending (FP32 squared distance, index).
// k-NN ranks, one query per lane: a CTA of KQ_WARPS warps serves 32 queries; warp w
// scans the candidates j = w, w + KQ_WARPS, ...  Every lane reads the same candidate
// row (a broadcast load), so the distance of one (query, candidate) pair costs a
// quarter of a float4 load, one subtraction and one fused multiply-add per
// coordinate.  Each lane keeps the exact top KNN_K of its candidates; the warps'
// lists are merged through shared memory at the end.
constexpr int KQ_WARPS = 4;

// Insert candidate j with squared-distance bits dk into the ascending list
// (D, I).  Candidates arrive in ascending j, so keeping an equal distance ahead
// of the newcomer orders the list by (distance, index).  Every position is
// updated from the old list at once (no chain of swaps).
__device__ __forceinline__ void knn_push(uint32_t (&D)[KNN_K], int (&I)[KNN_K], uint32_t dk, int j)
{
    if (dk < D[KNN_K - 1]) {
#pragma unroll
        for (int q = KNN_K - 1; q > 0; --q) {
            const bool shift = D[q - 1] > dk;
            const bool here = D[q] > dk;
            D[q] = shift ? D[q - 1] : (here ? dk : D[q]);
            I[q] = shift ? I[q - 1] : (here ? j : I[q]);
        }
        if (D[0] > dk) {
            D[0] = dk;
            I[0] = j;
        }
    }
}

__device__ __forceinline__ unsigned long long knn_key(uint32_t dk, int j)
{
    return (j < 0) ? ~0ull : (((unsigned long long)dk << 32) | (unsigned)j);
}

// Squared distance in coordinate order: each squared difference is added with
// a correctly rounded fused multiply-add (the oracle uses C's fmaf).
__device__ __forceinline__ float sqdist_rn(const float *a, const float *b, int d)
{
    float s = 0.f;
    for (int t = 0; t < d; ++t) {
        const float df = __fsub_rn(a[t], b[t]);
        s = __fmaf_rn(df, df, s);
    }
    return s;
}

constexpr int KQ_TILE = 128;
static_assert(KQ_TILE == KQ_WARPS * 32, "one tile row per thread in the compaction");
constexpr int KQ_MSTRIDE = KNN_K + 1;  // merge-list stride per lane (u64): spreads the banks

// Labels of the points, read from a byte copy in shared memory when the run is
// small enough (n <= KQ_LAB_CAP), else from global memory.
constexpr int KQ_LAB_CAP = 4096;
struct LabelView {
    const int *g;
    const unsigned char *s;
    bool in_smem;
    __device__ __forceinline__ int operator()(int j) const { return in_smem ? (int)s[j] : g[j]; }
};

// Cluster sizes from the labels (every CTA counts them itself: n reads); the
// labels are kept in shared memory on the way when they fit.
__device__ LabelView knn_label_counts(int n, const int *label, int *s_cnt /* [CMAX] */,
                                      unsigned char *s_lab /* [KQ_LAB_CAP] */)
{
    const bool keep = n <= KQ_LAB_CAP;
    if (threadIdx.x < CMAX) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int l = label[i];
        atomicAdd(&s_cnt[l], 1);
        if (keep) s_lab[i] = (unsigned char)l;
    }
    __syncthreads();
    return LabelView{label, s_lab, keep};
}

// Queries of one CTA, grouped by label.  The n points are ordered by (label,
// index); CTA b takes positions [32 b, 32 b + 32) of that order, so its queries
// come from one or two clusters and it scans only candidates with those labels.
// q_slot[32] receives the query indices (-1 past n); returns the label set as a
// bit mask.  s_cnt: the label counts.
__device__ unsigned long long knn_block_queries(int n, LabelView lab, int *q_slot, const int *s_cnt,
                                                int *s_wsum /* [KQ_WARPS] */)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 32) q_slot[tid] = -1;
    __syncthreads();
    const int p0 = blockIdx.x * 32, p1 = min(p0 + 32, n);
    unsigned long long mask = 0;
    int off = 0;
    for (int c = 0; c < CMAX; ++c) {
        const int cnt = s_cnt[c];
        const int lo = max(p0, off), hi = min(p1, off + cnt);
        if (lo < hi) {
            mask |= 1ull << c;
            // ranks [lo - off, hi - off) of label c, by ascending index
            const int r0 = lo - off, r1 = hi - off;
            int base = 0;
            for (int i0 = 0; i0 < n && base < r1; i0 += blockDim.x) {
                const int i = i0 + tid;
                const bool f = (i < n) && lab(i) == c;
                const unsigned bal = __ballot_sync(0xffffffffu, f);
                if (lane == 0) s_wsum[warp] = __popc(bal);
                __syncthreads();
                int before = base;
                for (int w2 = 0; w2 < warp; ++w2) before += s_wsum[w2];
                if (f) {
                    const int rk = before + __popc(bal & ((1u << lane) - 1u));
                    if (rk >= r0 && rk < r1) q_slot[off + rk - p0] = i;
                }
                int tot = 0;
                for (int w2 = 0; w2 < KQ_WARPS; ++w2) tot += s_wsum[w2];
                __syncthreads();
                base += tot;
            }
        }
        off += cnt;
    }
    __syncthreads();
    return mask;
}

// Merge the KQ_WARPS sorted lists of each lane's query (warp 0) and write ranks 1..KNN_K.
__device__ __forceinline__ void knn_merge_write(const unsigned long long *merge, bool act, int i, int *nbr)
{
    const int lane = threadIdx.x & 31;
    if ((threadIdx.x >> 5) != 0) return;
    int pos[KQ_WARPS];
#pragma unroll
    for (int w2 = 0; w2 < KQ_WARPS; ++w2) pos[w2] = 0;
    for (int rnk = 0; rnk < KNN_K; ++rnk) {
        unsigned long long best = ~0ull;
        int bw = 0;
#pragma unroll
        for (int w2 = 0; w2 < KQ_WARPS; ++w2) {
            const unsigned long long v = (pos[w2] < KNN_K) ? merge[(w2 * 32 + lane) * KQ_MSTRIDE + pos[w2]] : ~0ull;
            if (v < best) {
                best = v;
                bw = w2;
            }
        }
#pragma unroll
        for (int w2 = 0; w2 < KQ_WARPS; ++w2)
            if (w2 == bw) ++pos[w2];
        if (act) nbr[(long)i * KNN_K + rnk] = (best == ~0ull) ? -1 : (int)(best & 0xffffffffu);
    }
}

// Asynchronous global -> shared copies for the candidate tiles: 16 bytes with a
// zero fill past src_bytes (4, 8, 12 or 16), or one float.
__device__ __forceinline__ void cp_async16_fill(float *dst_smem, const float *src_gmem, int src_bytes)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src_gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(float *dst_smem, const float *src_gmem)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
// QR: query components held in registers (d <= QR, QR a multiple of 4).  The
// candidates whose label is one of the CTA's stream through shared memory in
// tiles (compacted, ascending index); every lane of a warp then reads the same
// row (a broadcast), two candidates at a time for independent accumulation
// chains.  Tiles are double-buffered: the rows of tile t + 1 are copied
// asynchronously (cp.async) while tile t is scanned.

template <int QR>
__device__ void knn_lanes(const float *x, int xstride, int n, int d, LabelView lab, const int *csize, int *nbr,
                          unsigned long long *merge /* [KQ_WARPS][32][KQ_MSTRIDE] */,
                          float *tile /* [2][KQ_TILE][QR], the same memory as merge */,
                          int *tidx /* [2][KQ_TILE] */, int *tlab /* [2][KQ_TILE] */, int *q_slot /* [32] */,
                          int *s_wsum /* [KQ_WARPS] */)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long lmask = knn_block_queries(n, lab, q_slot, csize, s_wsum);
    const int i = q_slot[lane];
    const bool act = i >= 0;
    const int li = act ? lab(i) : -1;
    const bool need = act && csize[li] >= 3;
    const bool any_need = __syncthreads_or(need);
    float q[QR];
#pragma unroll
    for (int t = 0; t < QR; ++t) q[t] = (act && t < d) ? x[(long)i * xstride + t] : 0.f;
    uint32_t Dl[KNN_K];
    int Il[KNN_K];
#pragma unroll
    for (int u = 0; u < KNN_K; ++u) {
        Dl[u] = 0xffffffffu;
        Il[u] = -1;
    }
    if (any_need) {
        const bool vec = ((reinterpret_cast<size_t>(x) & 15u) == 0) && (xstride & 3) == 0;
        // Compact the candidates [j0, j0 + KQ_TILE) whose label belongs to the CTA into
        // buffer b and start the copies of their rows (zeros past d, and in the row past
        // the last, which keeps the pair loop inside the tile).  Returns the row count.
        auto stage = [&](int j0, int b) -> int {
            const int jj = j0 + threadIdx.x;  // KQ_TILE == blockDim.x
            const int lj = (jj < n) ? lab(jj) : -1;
            const bool f = lj >= 0 && ((lmask >> lj) & 1ull);
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (lane == 0) s_wsum[warp] = __popc(bal);
            __syncthreads();  // also: buffer b (the tile before the previous one) is no longer read
            int pos = __popc(bal & ((1u << lane) - 1u)), rows = 0;
            for (int w2 = 0; w2 < KQ_WARPS; ++w2) {
                pos += (w2 < warp) ? s_wsum[w2] : 0;
                rows += s_wsum[w2];
            }
            int *ti = tidx + b * KQ_TILE;
            if (f) {
                ti[pos] = jj;
                tlab[b * KQ_TILE + pos] = lj;
            }
            __syncthreads();
            float *tb = tile + b * KQ_TILE * QR;
            const int rows2 = min(rows + 1, KQ_TILE);
            if (vec) {
                for (int e = threadIdx.x; e < rows2 * (QR / 4); e += blockDim.x) {
                    const int rr = e / (QR / 4), t4 = (e - rr * (QR / 4)) * 4;
                    float *dst = tb + rr * QR + t4;
                    const int bytes = (rr < rows) ? 4 * max(0, min(d - t4, 4)) : 0;
                    if (bytes > 0) cp_async16_fill(dst, x + (long)ti[rr] * xstride + t4, bytes);
                    else *reinterpret_cast<float4 *>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            } else {
                for (int e = threadIdx.x; e < rows2 * QR; e += blockDim.x) {
                    const int rr = e / QR, t = e - rr * QR;
                    float *dst = tb + rr * QR + t;
                    if (rr < rows && t < d) cp_async4(dst, x + (long)ti[rr] * xstride + t);
                    else *dst = 0.f;
                }
            }
            cp_async_commit();
            return rows;
        };
        int rows = stage(0, 0);
        for (int t = 0, j0 = 0; j0 < n; ++t, j0 += KQ_TILE) {
            const int b = t & 1;
            int rows_next = 0;
            if (j0 + KQ_TILE < n) rows_next = stage(j0 + KQ_TILE, b ^ 1);
            else cp_async_commit();  // an empty group keeps the wait below uniform
            cp_async_wait_prev();    // this thread's copies of tile t have landed
            __syncthreads();         // ... and every thread's
            const float *tb = tile + b * KQ_TILE * QR;
            const int *ti = tidx + b * KQ_TILE, *tl = tlab + b * KQ_TILE;
            for (int rr = warp * 2; rr < rows; rr += 2 * KQ_WARPS) {
                const float *ra = tb + rr * QR;
                const float *rb = tb + (rr + 1) * QR;  // inside the tile (zeros past the rows)
                float sa = 0.f, sb = 0.f;
#pragma unroll
                for (int t4 = 0; t4 < QR; t4 += 4) {
                    const float4 va = *reinterpret_cast<const float4 *>(ra + t4);
                    const float4 vb = *reinterpret_cast<const float4 *>(rb + t4);
                    float da = __fsub_rn(q[t4], va.x), db = __fsub_rn(q[t4], vb.x);
                    sa = __fmaf_rn(da, da, sa);
                    sb = __fmaf_rn(db, db, sb);
                    da = __fsub_rn(q[t4 + 1], va.y);
                    db = __fsub_rn(q[t4 + 1], vb.y);
                    sa = __fmaf_rn(da, da, sa);
                    sb = __fmaf_rn(db, db, sb);
                    da = __fsub_rn(q[t4 + 2], va.z);
                    db = __fsub_rn(q[t4 + 2], vb.z);
                    sa = __fmaf_rn(da, da, sa);
                    sb = __fmaf_rn(db, db, sb);
                    da = __fsub_rn(q[t4 + 3], va.w);
                    db = __fsub_rn(q[t4 + 3], vb.w);
                    sa = __fmaf_rn(da, da, sa);
                    sb = __fmaf_rn(db, db, sb);
                }
                const int ja = ti[rr];
                if (need && tl[rr] == li && ja != i) knn_push(Dl, Il, __float_as_uint(sa), ja);
                if (rr + 1 < rows) {
                    const int jb = ti[rr + 1];
                    if (need && tl[rr + 1] == li && jb != i) knn_push(Dl, Il, __float_as_uint(sb), jb);
                }
            }
            rows = rows_next;
        }
        __syncthreads();  // the merge lists below reuse the tile memory
    }
#pragma unroll
    for (int u = 0; u < KNN_K; ++u) merge[(warp * 32 + lane) * KQ_MSTRIDE + u] = knn_key(Dl[u], Il[u]);
    __syncthreads();
    knn_merge_write(merge, act, i, nbr);
}

// Queries wider than the register budget: the query row is read from global memory.
__device__ void knn_lanes_wide(const float *x, int xstride, int n, int d, LabelView lab, const int *csize, int *nbr,
                               unsigned long long *merge)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 32 + lane;
    const bool act = i < n;
    const int li = act ? lab(i) : -1;
    const bool need = act && csize[li] >= 3;
    const float *qi = x + (long)(act ? i : 0) * xstride;
    uint32_t Dl[KNN_K];
    int Il[KNN_K];
#pragma unroll
    for (int u = 0; u < KNN_K; ++u) {
        Dl[u] = 0xffffffffu;
        Il[u] = -1;
    }
    if (__any_sync(0xffffffffu, need)) {
        for (int j = warp; j < n; j += KQ_WARPS) {
            const int lj = lab(j);
            const float s = sqdist_rn(qi, x + (long)j * xstride, d);
            if (need && lj == li && j != i) knn_push(Dl, Il, __float_as_uint(s), j);
        }
    }
#pragma unroll
    for (int u = 0; u < KNN_K; ++u) merge[(warp * 32 + lane) * KQ_MSTRIDE + u] = knn_key(Dl[u], Il[u]);
    __syncthreads();
    knn_merge_write(merge, act, i, nbr);
}

// Register width of the query for dimension d (0: the wide form).
__host__ __device__ constexpr int knn_qr(int d) { return d <= 8 ? 8 : d <= 16 ? 16 : d <= 32 ? 32 : d <= 64 ? 64 : 0; }
// Bytes of the region shared by the merge lists and the two candidate tiles.
__host__ __device__ constexpr size_t knn_region_bytes(int d)
{
    return (sizeof(unsigned long long) * KQ_WARPS * 32 * KQ_MSTRIDE > sizeof(float) * 2 * KQ_TILE * knn_qr(d))
               ? sizeof(unsigned long long) * KQ_WARPS * 32 * KQ_MSTRIDE
               : sizeof(float) * 2 * KQ_TILE * knn_qr(d);
}

// shared memory: merge lists [KQ_WARPS][32][KQ_MSTRIDE] u64, in the same memory as the candidate tiles
// [2][KQ_TILE][QR] f32 | tile indices and labels [2][KQ_TILE] each | query slots [32] | label counts
// [CMAX] | warp sums [KQ_WARPS] | labels as bytes [KQ_LAB_CAP].  The cluster sizes come from the labels
// themselves, so the k-NN may run while the statistics are being updated.
__device__ void knn_rows(const float *x, int xstride, int n, int d, const int *label, int *nbr, float *smem)
{
    unsigned long long *merge = reinterpret_cast<unsigned long long *>(smem);
    float *tile = smem;
    int *tidx = reinterpret_cast<int *>(reinterpret_cast<char *>(smem) + knn_region_bytes(d));
    int *tlab = tidx + 2 * KQ_TILE;
    int *q_slot = tlab + 2 * KQ_TILE;
    int *s_cnt = q_slot + 32;
    int *s_wsum = s_cnt + CMAX;
    unsigned char *s_lab = reinterpret_cast<unsigned char *>(s_wsum + KQ_WARPS);
    const LabelView lab = knn_label_counts(n, label, s_cnt, s_lab);
    if (d <= 8) knn_lanes<8>(x, xstride, n, d, lab, s_cnt, nbr, merge, tile, tidx, tlab, q_slot, s_wsum);
    else if (d <= 16) knn_lanes<16>(x, xstride, n, d, lab, s_cnt, nbr, merge, tile, tidx, tlab, q_slot, s_wsum);
    else if (d <= 32) knn_lanes<32>(x, xstride, n, d, lab, s_cnt, nbr, merge, tile, tidx, tlab, q_slot, s_wsum);
    else if (d <= 64) knn_lanes<64>(x, xstride, n, d, lab, s_cnt, nbr, merge, tile, tidx, tlab, q_slot, s_wsum);
    else knn_lanes_wide(x, xstride, n, d, lab, s_cnt, nbr, merge);
}

__global__ void __launch_bounds__(KQ_WARPS * 32) k_knn(DevCtx C, int r0)
{
    extern __shared__ float ksm[];
    const int r = r0 + blockIdx.y;
    const RunDesc &D = C.desc[r];
    if (C.state[r].done || !D.clustering) return;
    const int d = D.d;
    knn_rows(C.fa + D.x_off, D.d_pad, D.n_live, d, C.label + D.pt_off, C.nbr + D.nbr_off, ksm);
}

size_t knn_smem_bytes(int d)
{
    // the region for the widest register form also covers every narrower run and the wide form
    return knn_region_bytes(d < 64 ? d : 64) + sizeof(int) * (4 * KQ_TILE + 32 + CMAX + KQ_WARPS) + KQ_LAB_CAP;
}

// Union-find in shared memory: roots are the smallest member index.
__device__ __forceinline__ int uf_find(volatile int *par, int x)
{
    for (;;) {
        const int p = par[x];
        if (p == x) return x;
        const int gp = par[p];
        if (gp != p) par[x] = gp;
        x = p;
    }
}
__device__ __forceinline__ bool uf_union(int *par, int a, int b)
{
    for (;;) {
        a = uf_find(par, a);
        b = uf_find(par, b);
        if (a == b) return false;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(&par[b], b, a);
        if (old == b) return true;
        b = old;
    }
}

// The (rank)-th neighbour of point i when the precomputed ranks are exhausted:
// the smallest (distance, index) key above `prev` among same-label points.
__device__ unsigned long long next_neighbour(const float *x, int xstride, int n, int d, const int *label, int i,
                                             unsigned long long prev)
{
    unsigned long long best = ~0ull;
    const int li = label[i];
    for (int j = 0; j < n; ++j) {
        if (j == i || label[j] != li) continue;
        const float s = sqdist_rn(x + (long)i * xstride, x + (long)j * xstride, d);
        const unsigned long long key = ((unsigned long long)__float_as_uint(s) << 32) | (unsigned)j;
        if (key > prev && key < best) best = key;
    }
    return best;
}

// Components of the k-NN graphs of every active cluster (Algorithm 4): ranks 1
// and 2 first, then rank k = 3, 4, ... until a rank merges nothing in that
// cluster or the ranks are exhausted (k > m - 1).  Writes comp[i] = root.
// par: shared [n]; lastkey: global scratch [n] for ranks beyond KNN_K.
__device__ void knn_components_block(const float *x, int xstride, int n, int d, const int *label,
                                     const int *csize, int *active, const int *nbr, int *par,
                                     unsigned long long *lastkey, int *s_merged, int *s_live)
{
    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += blockDim.x) par[i] = i;
    __syncthreads();
    for (int rank = 1;; ++rank) {
        if (tid < CMAX) s_merged[tid] = 0;
        if (tid == 0) *s_live = 0;
        __syncthreads();
        for (int i = tid; i < n; i += blockDim.x) {
            const int c = label[i];
            if (!active[c] || rank > csize[c] - 1) continue;
            int j;
            if (rank <= KNN_K) {
                j = nbr[(long)i * KNN_K + rank - 1];
                if (rank == KNN_K && j >= 0) {
                    const float s = sqdist_rn(x + (long)i * xstride, x + (long)j * xstride, d);
                    lastkey[i] = ((unsigned long long)__float_as_uint(s) << 32) | (unsigned)j;
                }
            } else {
                const unsigned long long key = next_neighbour(x, xstride, n, d, label, i, lastkey[i]);
                lastkey[i] = key;
                j = (key == ~0ull) ? -1 : (int)(key & 0xffffffffu);
            }
            if (j >= 0 && uf_union(par, i, j)) s_merged[c] = 1;
        }
        __syncthreads();
        if (tid < CMAX && active[tid]) {
            // a cluster stops at the first rank k >= 3 that merges nothing (its
            // component sizes repeat), or once its ranks are exhausted (k = m - 1)
            const bool stop = (rank >= 3 && !s_merged[tid]) || rank >= csize[tid] - 1;
            if (stop) active[tid] = 0;
            else atomicAdd(s_live, 1);
        }
        __syncthreads();
        const int live = *s_live;
        __syncthreads();
        if (live == 0) break;
    }
    for (int i = tid; i < n; i += blockDim.x) par[i] = uf_find(par, i);
    __syncthreads();
}

__device__ void stats_split(Stats *st, int p, int np, const int *sz, const int *ids)
{
    // eqs. new0-new6; new3 for Y in {Z, X_q} over every other live cluster q
    const double n = (double)st->n[p];
    const double Xp = st->logXp[p], Xp2 = st->logXp2[p], Zp = st->logZp[p], Zp2 = st->logZp2[p];
    const double ZXp = st->logZXp[p], ZpXp = st->logZpXp[p];
    double XXold[CMAX];
    int others[CMAX];
    for (int q = 0; q < CMAX; ++q) {
        XXold[q] = st->logXX[p * CMAX + q];
        others[q] = st->alive[q] && q != p;
    }
    for (int i = 0; i < np; ++i) {
        const int c = ids[i];
        const double ni = (double)sz[i];
        const double fi = log(ni) - log(n);
        const double gi = log(ni) + log(ni + 1.0) - log(n) - log(n + 1.0);
        st->alive[c] = 1;
        st->n[c] = sz[i];
        st->logXp[c] = fi + Xp;
        st->logXp2[c] = gi + Xp2;
        st->logZXp[c] = fi + ZXp;
        st->logZp[c] = fi + Zp;
        st->logZpXp[c] = gi + ZpXp;
        st->logZp2[c] = gi + Zp2;
    }
    for (int i = 0; i < np; ++i) {
        const int c = ids[i];
        const double fi = log((double)sz[i]) - log(n);
        for (int q = 0; q < CMAX; ++q) {
            if (!others[q]) continue;
            st->logXX[c * CMAX + q] = fi + XXold[q];
            st->logXX[q * CMAX + c] = fi + XXold[q];
        }
        for (int j = 0; j < np; ++j) {
            if (j == i) continue;
            st->logXX[c * CMAX + ids[j]] = log((double)sz[i]) + log((double)sz[j]) - log(n) - log(n + 1.0) + Xp2;
        }
    }
}

constexpr int CL_THREADS = 1024;

__device__ void cluster_body(DevCtx C, unsigned long long *lastkey_all, int r, int *csm)
{
    const RunDesc &D = C.desc[r];
    RunState *S = C.state + r;
    if (S->done || !D.clustering) return;
    Stats *st = C.stats + r;
    const int n = D.n_live;
    int *par = csm;          // [n] union-find parents, then component roots
    int *cnt = csm + n;      // [n] component sizes by root, then new ids by root
    int *lab = csm + 2 * n;  // [n] labels (shared copy)
    __shared__ int s_active[CMAX], s_csize[CMAX], s_merged[CMAX], s_live[1 + CMAX], s_fail;
    __shared__ int s_nroots[CMAX], s_split[CMAX], s_nsplit;
    __shared__ int s_roots[CMAX * CMAX];  // ascending roots of the clusters that split
    __shared__ int s_wsum[CL_THREADS / 32];
    const int tid = threadIdx.x;
    int *label = C.label + D.pt_off;
    for (int i = tid; i < n; i += blockDim.x) lab[i] = label[i];
    if (tid < CMAX) {
        s_csize[tid] = st->alive[tid] ? st->n[tid] : 0;
        s_active[tid] = st->alive[tid] && st->n[tid] >= 3;
        s_nroots[tid] = 0;
        s_split[tid] = 0;
    }
    if (tid == 0) {
        s_fail = 0;
        s_nsplit = 0;
    }
    __syncthreads();
    knn_components_block(C.fa + D.x_off, D.d_pad, n, D.d, lab, s_csize, s_active, C.nbr + D.nbr_off, par,
                         lastkey_all + D.pt_off, s_merged, s_live);
    // component sizes and the number of components of every cluster
    for (int i = tid; i < n; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
        atomicAdd(&cnt[par[i]], 1);
        if (par[i] == i) atomicAdd(&s_nroots[lab[i]], 1);
    }
    __syncthreads();
    // clusters that split (ascending id; only clusters present at the start of the iteration)
    if (tid == 0) {
        int ns = 0;
        for (int c = 0; c < CMAX; ++c)
            if (st->alive[c] && s_csize[c] >= 3 && s_nroots[c] > 1) {
                if (s_nroots[c] > CMAX) s_fail = 1;
                s_split[ns++] = c;
            }
        s_nsplit = ns;
    }
    __syncthreads();
    const int nsplit = s_nsplit;
    if (nsplit > 0 && !s_fail) {
        // ascending roots of each splitting cluster: an ordered block-wide compaction
        for (int q = 0; q < nsplit; ++q) {
            const int c = s_split[q];
            int base = 0;
            for (int i0 = 0; i0 < n; i0 += blockDim.x) {
                const int i = i0 + tid;
                const int f = (i < n && lab[i] == c && par[i] == i) ? 1 : 0;
                const unsigned bal = __ballot_sync(0xffffffffu, f);
                const int lane = tid & 31, warp = tid >> 5;
                if (lane == 0) s_wsum[warp] = __popc(bal);
                __syncthreads();
                int off = base;
                for (int w2 = 0; w2 < warp; ++w2) off += s_wsum[w2];
                if (f) {
                    const int pos = off + __popc(bal & ((1u << lane) - 1u));
                    if (pos < CMAX) s_roots[q * CMAX + pos] = i;
                }
                int tot = 0;
                for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) tot += s_wsum[w2];
                __syncthreads();
                base += tot;
            }
        }
        __syncthreads();
        if (tid == 0) {
            // split in ascending id order: part 0 (smallest member) keeps the id, the
            // others take the lowest free ids (Algorithm 3, eqs. new0-new6)
            for (int q = 0; q < nsplit && !s_fail; ++q) {
                const int c = s_split[q];
                const int np = s_nroots[c];
                int sz[CMAX], ids[CMAX];
                for (int pi = 0; pi < np; ++pi) sz[pi] = cnt[s_roots[q * CMAX + pi]];
                ids[0] = c;
                int nxt = 0;
                for (int pi = 1; pi < np; ++pi) {
                    while (nxt < CMAX && (st->alive[nxt] || nxt == c)) ++nxt;
                    if (nxt >= CMAX) {
                        s_fail = 1;
                        break;
                    }
                    ids[pi] = nxt++;
                }
                if (s_fail) break;
                stats_split(st, c, np, sz, ids);
                for (int pi = 0; pi < np; ++pi) cnt[s_roots[q * CMAX + pi]] = ids[pi];
            }
        }
        __syncthreads();
        if (!s_fail) {
            for (int i = tid; i < n; i += blockDim.x) {
                const int c = lab[i];
                bool sp = false;
                for (int q = 0; q < nsplit; ++q) sp |= (s_split[q] == c);
                if (sp) label[i] = cnt[par[i]];
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (s_fail) {
            S->status = NS_ERR_CAPACITY;
            S->done = 1;
            S->final_done = 1;
        }
        int na = 0;
        for (int c = 0; c < CMAX; ++c) na += st->alive[c];
        S->n_clusters = na;
        if (na > S->max_clusters) S->max_clusters = na;
    }
}

// Termination test of the previous iteration, cluster finding and selection of this
// one, for one run per CTA: one launch instead of three on the iteration's path.
static_assert(CL_THREADS == SORT_THREADS, "one block shape");
__global__ void __launch_bounds__(SORT_THREADS) k_term_cluster_sort(DevCtx C, unsigned long long *lastkey_all, int r0,
                                                                  int do_term, int clustering)
{
    extern __shared__ unsigned char fsm[];
    const int r = r0 + blockIdx.x;
    if (do_term && threadIdx.x == 0) term_body(C, r);
    __syncthreads();
    if (clustering) {
        cluster_body(C, lastkey_all, r, reinterpret_cast<int *>(fsm));
        __syncthreads();
    }
    sort_body(C, r, fsm);
}

size_t cluster_smem_bytes(int n_live_max) { return sizeof(int) * 3 * (size_t)n_live_max; }

// ------------------------------------------------------------------------
// Posterior statistics: H = sum_i p_i (log L_i - log Z), one CTA per run.
// ------------------------------------------------------------------------
__global__ void k_info(DevCtx C, int r, double logz, double *part)
{
    const RunDesc &D = C.desc[r];
    const long n = C.state[r].n_dead;
    __shared__ double sh[32], sp[32];
    double h = 0.0, ps = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        if (!gg_in(i, D.dead_cap, C.state + r)) break;
        const double ll = (double)D.dead_logl[D.dead_off + i];
        const double lp = D.dead_logw[D.dead_off + i] + ll - logz;
        const double p = exp(lp);
        if (p > 0.0) {
            h += p * (ll - logz);
            ps += p;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        h += __shfl_xor_sync(0xffffffffu, h, o);
        ps += __shfl_xor_sync(0xffffffffu, ps, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[threadIdx.x >> 5] = h;
        sp[threadIdx.x >> 5] = ps;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[w];
            b += sp[w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// ------------------------------------------------------------------------
// Component entry-point kernels
// ------------------------------------------------------------------------
__global__ void k_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, long n)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const U4 c{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    const U4 o = philox4x32_10(c, k0, k1);
    out[4 * i] = o.x;
    out[4 * i + 1] = o.y;
    out[4 * i + 2] = o.z;
    out[4 * i + 3] = o.w;
}

__global__ void __launch_bounds__(SEL_THREADS) k_sort_logl(const float *logl, int n, int *order)
{
    extern __shared__ unsigned long long skeys[];
    const int npow = next_pow2(n);
    for (int i = threadIdx.x; i < npow; i += blockDim.x)
        skeys[i] = (i < n) ? ((unsigned long long)float_key(logl[i]) << 32) | (unsigned)i : ~0ull;
    __syncthreads();
    block_bitonic_sort(skeys, npow);
    for (int i = threadIdx.x; i < n; i += blockDim.x) order[i] = (int)(skeys[i] & 0xffffffffu);
}

__global__ void __launch_bounds__(KQ_WARPS * 32) k_knn_plain(const float *x, int n, int d, const int *label, int *nbr)
{
    extern __shared__ float ksm[];
    knn_rows(x, d, n, d, label, nbr, ksm);
}

__global__ void __launch_bounds__(CL_THREADS) k_components_plain(const float *x, int n, int d, const int *label,
                                                                 const int *csize_g, const int *nbr, int *comp,
                                                                 unsigned long long *lastkey, int *ncomp)
{
    extern __shared__ int csm[];
    __shared__ int s_active[CMAX], s_csize[CMAX], s_merged[CMAX], s_live[1 + CMAX];
    if (threadIdx.x < CMAX) {
        s_csize[threadIdx.x] = csize_g[threadIdx.x];
        s_active[threadIdx.x] = csize_g[threadIdx.x] >= 3;
    }
    __syncthreads();
    knn_components_block(x, d, n, d, label, s_csize, s_active, nbr, csm, lastkey, s_merged, s_live);
    for (int i = threadIdx.x; i < n; i += blockDim.x) comp[i] = csm[i];
    if (threadIdx.x == 0) {
        int c = 0;
        for (int i = 0; i < n; ++i) c += (csm[i] == i);
        *ncomp = c;
    }
}

__global__ void __launch_bounds__(SEL_THREADS) k_stats_plain(Stats *st, double *zz, int k, const double *kL,
                                                             const int *kP, double *logw_out)
{
    extern __shared__ unsigned char sraw[];
    EvScratch *E = reinterpret_cast<EvScratch *>(sraw);
    evidence_batch(st, &zz[0], &zz[1], k, kL, kP, E);
    for (int j = threadIdx.x; j < k; j += blockDim.x) logw_out[j] = E->logw[kP[j]];
}

size_t evscratch_bytes() { return sizeof(EvScratch); }

}  // namespace ggns

// ------------------------------------------------------------------------
// Export of weighted samples: x (FP64, unpadded) and log p_i = log w_i + log L_i - log Z.
// ------------------------------------------------------------------------
namespace ggns {

__global__ void k_export(DevCtx C, int r, int d, int d_pad, double logz, double *x, double *logp, long n)
{
    const RunDesc &D = C.desc[r];
    const long tot = n * d;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
        const long i = e / d, c = e % d;
        if (!gg_in(i, D.dead_cap, C.state + r)) break;
        if (x) x[e] = (double)D.dead_x[(D.dead_off + i) * d_pad + c];
        if (c == 0 && logp) logp[i] = D.dead_logw[D.dead_off + i] + (double)D.dead_logl[D.dead_off + i] - logz;
    }
}

__global__ void k_reduce_parts(const double *part, int n_parts, int len, double *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int p = 0; p < n_parts; ++p) s += part[(long)p * len + i];
        out[i] = s;
    }
}

// Opt a kernel in to `smem` bytes of dynamic shared memory when its static and
// dynamic shared memory together exceed the default 48 KiB.
static cudaError_t set_max_smem(const void *fn, size_t smem)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, fn);
    if (e != cudaSuccess) return e;
    if (smem + a.sharedSizeBytes > 48 * 1024)
        return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

cudaError_t prepare_iteration_kernels(size_t sel_smem, size_t knn_smem, size_t cl_smem, size_t sort_smem)
{
    cudaError_t e;
    if ((e = set_max_smem((const void *)k_evidence, sel_smem)) != cudaSuccess) return e;
    if ((e = set_max_smem((const void *)k_final, sel_smem)) != cudaSuccess) return e;
    if ((e = set_max_smem((const void *)k_knn, knn_smem)) != cudaSuccess) return e;
    return set_max_smem((const void *)k_term_cluster_sort, cl_smem > sort_smem ? cl_smem : sort_smem);
}

cudaError_t launch_evidence(const DevCtx &C, int r0, int n_runs, size_t smem, cudaStream_t s)
{
    k_evidence<<<n_runs, SEL_THREADS, smem, s>>>(C, r0);
    return cudaGetLastError();
}
cudaError_t launch_final(const DevCtx &C, int r0, int n_runs, size_t smem, cudaStream_t s)
{
    k_final<<<n_runs, SEL_THREADS, smem, s>>>(C, r0);
    return cudaGetLastError();
}
// Momentum noise of the single-pass HSS, drawn ahead of the walk (the same
// Philox blocks and Box-Muller pairs the walker would draw): one thread per
// (walker, step, block of four components).
constexpr int NOISE_THREADS = 256;

__global__ void __launch_bounds__(NOISE_THREADS) k_noise(DevCtx C, const int *run_list, RecView R, const long *rec_base)
{
    const int r = run_list[blockIdx.y];
    const RunDesc &D = C.desc[r];
    const RunState *S = C.state + r;
    if (S->done) return;
    if (D.d_pad & 3) return;      // drawn in the walk (no whole blocks of four components)
    const unsigned nb = (unsigned)(D.d_pad >> 2);  // blocks of four components
    const unsigned steps = (unsigned)noise_steps(R.nT, S->t_stop_last);
    // item = (walker, step, block); fewer than 2^32 (the noise buffer holds < 2^31 floats).
    // 32-bit index arithmetic, a shift where the block count is a power of two
    const unsigned items = (unsigned)D.k * steps * nb;
    const bool pow2 = (nb & (nb - 1u)) == 0u;
    const int sh = __ffs((int)nb) - 1;
    const uint32_t iter = (uint32_t)S->iter;
    const long wrow0 = rec_base[r] / R.rec_len;  // first walker row of this run
    for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        const unsigned ws = pow2 ? (it >> sh) : it / nb;
        const unsigned b = it - ws * nb;
        const unsigned w = ws / steps;
        const unsigned ts = ws - w * steps + 1u;
        const U4 wd = rng_block(D, iter, P_NOISE, w, ts, b);
        float4 z;
        box_muller(wd.x, wd.y, z.x, z.y);
        box_muller(wd.z, wd.w, z.z, z.w);
        const long row = (wrow0 + w) * R.nT + (ts - 1);
        *reinterpret_cast<float4 *>(R.nz + row * R.xs + 4 * b) = z;
        if (b == 0) R.nsp[row] = spare_bits(wd);
    }
}

cudaError_t launch_noise(const DevCtx &C, const int *runs, int nr, int blocks_per_run, const RecView &R,
                         const long *rec_base, cudaStream_t s)
{
    k_noise<<<dim3(blocks_per_run, nr), NOISE_THREADS, 0, s>>>(C, runs, R, rec_base);
    return cudaGetLastError();
}

cudaError_t launch_hss_pick(const DevCtx &C, const int *runs, int nr, int max_k, const RecView &R, const long *rec_base,
                            cudaStream_t s)
{
    k_hss_pick<<<dim3((max_k + PICK_WARPS - 1) / PICK_WARPS, nr), PICK_WARPS * 32, 0, s>>>(C, runs, R, rec_base);
    return cudaGetLastError();
}
cudaError_t launch_territory(const DevCtx &C, int r0, int n_runs, int max_k, int max_d, cudaStream_t s)
{
    const size_t smem = territory_smem_bytes(max_d);
    static size_t opted = 48 * 1024;
    if (smem > opted) {
        cudaError_t e = cudaFuncSetAttribute(k_territory, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        opted = smem;
    }
    k_territory<<<dim3((max_k + 31) / 32, n_runs), TER_WARPS * 32, smem, s>>>(C, r0);
    return cudaGetLastError();
}
cudaError_t launch_territory_plain(const float *surv, const int *surv_label, int m_s, const float *xn, const int *want,
                                   int k, int d, int *keep, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    const size_t smem = territory_smem_bytes(d);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_territory_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_territory_plain<<<(k + 31) / 32, TER_WARPS * 32, smem, s>>>(surv, surv_label, m_s, xn, want, k, d, keep);
    return cudaGetLastError();
}
cudaError_t launch_term_cluster_sort(const DevCtx &C, int r0, int n_runs, unsigned long long *lastkey, size_t smem,
                                     bool do_term, bool clustering, cudaStream_t s)
{
    k_term_cluster_sort<<<n_runs, SORT_THREADS, smem, s>>>(C, lastkey, r0, do_term ? 1 : 0, clustering ? 1 : 0);
    return cudaGetLastError();
}
cudaError_t launch_term(const DevCtx &C, int r0, int n_runs, cudaStream_t s)
{
    k_term<<<(n_runs + 127) / 128, 128, 0, s>>>(C, r0, n_runs);
    return cudaGetLastError();
}
cudaError_t launch_tail(const DevCtx &C, int r0, int n_runs, cudaStream_t s)
{
    k_tail<<<n_runs, 256, 0, s>>>(C, r0);
    return cudaGetLastError();
}
cudaError_t launch_knn(const DevCtx &C, int r0, int n_runs, int max_nlive, size_t smem, cudaStream_t s)
{
    dim3 grid((max_nlive + 31) / 32, n_runs);
    k_knn<<<grid, KQ_WARPS * 32, smem, s>>>(C, r0);
    return cudaGetLastError();
}
constexpr int INFO_BLOCKS = 152;
cudaError_t launch_info(const DevCtx &C, int r, double logz, double *out, cudaStream_t s)
{
    // out: [2] result followed by [2 * INFO_BLOCKS] partials
    k_info<<<INFO_BLOCKS, 256, 0, s>>>(C, r, logz, out + 2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_parts(out + 2, INFO_BLOCKS, 2, out, s);
}
cudaError_t launch_export(const DevCtx &C, int r, int d, int d_pad, double logz, double *x, double *logp, long n,
                          cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long blocks = (n * d + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_export<<<(int)blocks, 256, 0, s>>>(C, r, d, d_pad, logz, x, logp, n);
    return cudaGetLastError();
}
cudaError_t launch_reduce_parts(const double *part, int n_parts, int len, double *out, cudaStream_t s)
{
    k_reduce_parts<<<(len + 255) / 256, 256, 0, s>>>(part, n_parts, len, out);
    return cudaGetLastError();
}
cudaError_t launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctr, k0, k1, out, n);
    return cudaGetLastError();
}
cudaError_t launch_sort_logl(const float *logl, int n, int *order, cudaStream_t s)
{
    const size_t smem = (size_t)next_pow2(n) * 8;
    cudaError_t e = set_max_smem((const void *)k_sort_logl, smem);
    if (e != cudaSuccess) return e;
    k_sort_logl<<<1, SEL_THREADS, smem, s>>>(logl, n, order);
    return cudaGetLastError();
}
cudaError_t launch_knn_components(const float *x, int n, int d, const int *label, const int *csize, int *nbr,
                                  int *comp, unsigned long long *lastkey, int *ncomp, cudaStream_t s)
{
    const size_t ks = knn_smem_bytes(d);
    cudaError_t e = set_max_smem((const void *)k_knn_plain, ks);
    if (e != cudaSuccess) return e;
    k_knn_plain<<<(n + 31) / 32, KQ_WARPS * 32, ks, s>>>(x, n, d, label, nbr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t cs = sizeof(int) * (size_t)n;
    e = set_max_smem((const void *)k_components_plain, cs);
    if (e != cudaSuccess) return e;
    k_components_plain<<<1, CL_THREADS, cs, s>>>(x, n, d, label, csize, nbr, comp, lastkey, ncomp);
    return cudaGetLastError();
}
cudaError_t launch_stats_plain(Stats *st, double *zz, int k, const double *kL, const int *kP, double *logw,
                               cudaStream_t s)
{
    const size_t smem = sizeof(EvScratch);
    cudaError_t e = set_max_smem((const void *)k_stats_plain, smem);
    if (e != cudaSuccess) return e;
    k_stats_plain<<<1, SEL_THREADS, smem, s>>>(st, zz, k, kL, kP, logw);
    return cudaGetLastError();
}

}  // namespace ggns
