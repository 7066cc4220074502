/*
 * ggns_oracle.c -- plain, slow, single-threaded FP64 reference implementation of
 * gradient-guided nested sampling (GGNS, arXiv 2312.03911).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; it exists so that tests, the smoke check and the CPU-baseline leg of
 * the benchmark can compare the CUDA library against an independent statement of
 * the method.  It shares no code, header, table or constant generator with the
 * CUDA path.
 *
 * What it follows, step by step:
 *   - the nested-sampling driver of Algorithm 3 (the full GGNS loop);
 *   - the cluster finding of Algorithm 4 (k-nearest-neighbour components);
 *   - the batched Hamiltonian slice sampler of Algorithm 5 with the reflection
 *     p' = p - 2 (p.n) n of the reflection equation (Section 2.3);
 *   - the cluster summary statistics of Appendix H (eqs. ini0-ini11,
 *     update0-update9, new0-new6), kept in log space;
 *   - the evidence definition Z = int L pi dtheta and the importance weights
 *     p_i = L_i w_i / Z (Appendix A);
 *   - the XL-peak termination (Section 3, Appendix I) and the classic
 *     remaining-evidence termination (Algorithm 1);
 *   - the torus reward of Section 4 (eq. torus) on a periodic prior, whose
 *     normaliser Appendix F gives in closed form.
 * Readings of passages that are ambiguous or garbled: the initial momentum is
 * N(0, I); states are saved once every walker has reflected min_ref times and the
 * loop runs until every walker has reflected max_ref times (the global loop
 * condition of Algorithm 5); the momentum noise perturbs inside steps only and an
 * outside step only reflects (Section 2.3: a particle left behind the boundary
 * gets stuck); each walker returns one state drawn uniformly over the steps of the
 * saving window, and a drawn outside step is rejected, so the walker returns its
 * start point (the rejection of slice sampling, Section 2.3); with more than one
 * cluster alive, a new point whose nearest surviving point belongs to another
 * cluster is rejected the same way (a cluster's new points stay in its region);
 * the prior box reflects a walker exactly (the position folds back across the
 * face and the momentum component flips), so, as in Algorithm 5, only the
 * iso-likelihood boundary makes a step an outside step;
 * strict inequality L > L*; update6 read as ZX_q -> ZX_q + X_pX_q L/(n_p+1);
 * the final sweep with decreasing n_p; the XL-peak statistic taken on the
 * dead-point sequence, L_i X_i, as the hyper-parameter table of Appendix C
 * defines it.  The printed forms (noise on every step, the pick among saved
 * inside states only, no region check, the box as an outside region) remain
 * switches of orc_cfg_t.  An option, not the default: the time-reversible form of the
 * step (midpoint: half move, reflection with the normal at the half step, half move),
 * against which the printed step (move, then reflection at the new point) is compared.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written here from its published
 * definition, with the counter layout
 *     key     = (seed_lo, seed_hi ^ run_id)
 *     counter = (block, step, slot, (iteration << 4) | purpose).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no FMA contraction, so
 * that the FP32 k-NN distances round exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NEG_INF (-INFINITY)

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (SC'11 definition)                                           */
/* ------------------------------------------------------------------------- */

enum {
    ORC_P_INIT = 0,    /* prior draw of live point `slot`                     */
    ORC_P_MOM = 1,     /* initial momentum of walker `slot`                   */
    ORC_P_NOISE = 2,   /* momentum noise eps at step `step`                   */
    ORC_P_RES = 3,     /* reserved (the reservoir uses spare bits of the noise) */
    ORC_P_CLUSTER = 4, /* cluster choice of walker `slot`                     */
    ORC_P_START = 5,   /* start-point choice of walker `slot`                 */
    ORC_P_PRUNE = 6    /* fresh momentum after pruning at step `step`         */
};

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u; /* golden-ratio Weyl increment */
            k1 += 0xBB67AE85u; /* sqrt(3)-1 Weyl increment    */
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void orc_rng_block(uint64_t seed, uint32_t run_id, uint32_t iter, uint32_t purpose,
                          uint32_t slot, uint32_t step, uint32_t block, uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ run_id};
    uint32_t ctr[4] = {block, step, slot, (iter << 4) | (purpose & 15u)};
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform in (0,1): the top 23 bits plus one half, times 2^-23.  Exact in FP32 and FP64. */
static double orc_u01(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

/* FP64 uniform in (0,1) from two words: 52 bits plus one half, times 2^-52. */
static double orc_u01_53(uint32_t r0, uint32_t r1)
{
    uint64_t m = ((uint64_t)r0 << 20) | (uint64_t)(r1 >> 12);
    return ((double)m + 0.5) * (1.0 / 4503599627370496.0);
}

/* d standard normals by Box-Muller: block b gives components 4b..4b+3 from
 * (u0,u1) -> (r cos 2 pi u1, r sin 2 pi u1), r = sqrt(-2 ln u0), and likewise (u2,u3). */
void orc_normals(uint64_t seed, uint32_t run_id, uint32_t iter, uint32_t purpose,
                 uint32_t slot, uint32_t step, int d, double *z)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int b = 0; 4 * b < d; ++b) {
        uint32_t w[4];
        orc_rng_block(seed, run_id, iter, purpose, slot, step, (uint32_t)b, w);
        double ra = sqrt(-2.0 * log(orc_u01(w[0])));
        double rb = sqrt(-2.0 * log(orc_u01(w[2])));
        double v[4] = {ra * cos(two_pi * orc_u01(w[1])), ra * sin(two_pi * orc_u01(w[1])),
                       rb * cos(two_pi * orc_u01(w[3])), rb * sin(two_pi * orc_u01(w[3]))};
        for (int i = 0; i < 4 && 4 * b + i < d; ++i) z[4 * b + i] = v[i];
    }
}

/* ------------------------------------------------------------------------- */
/* Likelihood families and their gradients (the score, Section 2.3)           */
/* ------------------------------------------------------------------------- */

enum { ORC_LIK_ISO = 0, ORC_LIK_MIX_ISO = 1, ORC_LIK_DENSE = 2, ORC_LIK_DENSE_MIX = 3, ORC_LIK_ROSEN = 4,
       ORC_LIK_TORUS = 5 };

typedef struct {
    int kind;
    int d;
    int n_comp;
    const double *means;       /* [n_comp][d]                          */
    const double *log_weights; /* [n_comp]; NULL means equal weights   */
    const double *sigma;       /* [n_comp] isotropic standard deviation */
    const double *precision;   /* [d][d], symmetric positive definite   */
    double rosen_scale;        /* multiplies the Rosenbrock sum         */
    double torus_alpha, torus_beta, torus_c; /* torus reward (Section 4, eq. torus) */
} orc_lik_t;

/* log det of an SPD matrix by an unpivoted Cholesky factorisation; NAN if not SPD. */
double orc_logdet_spd(int d, const double *a)
{
    double *l = (double *)calloc((size_t)d * d, sizeof(double));
    double logdet = 0.0;
    for (int j = 0; j < d; ++j) {
        double s = a[(size_t)j * d + j];
        for (int k = 0; k < j; ++k) s -= l[(size_t)j * d + k] * l[(size_t)j * d + k];
        if (!(s > 0.0)) { free(l); return NAN; }
        double ljj = sqrt(s);
        l[(size_t)j * d + j] = ljj;
        logdet += 2.0 * log(ljj);
        for (int i = j + 1; i < d; ++i) {
            double t = a[(size_t)i * d + j];
            for (int k = 0; k < j; ++k) t -= l[(size_t)i * d + k] * l[(size_t)j * d + k];
            l[(size_t)i * d + j] = t / ljj;
        }
    }
    free(l);
    return logdet;
}

static double orc_comp_logw(const orc_lik_t *lk, int k)
{
    return lk->log_weights ? lk->log_weights[k] : -log((double)lk->n_comp);
}

/* log L(x) and, if grad != NULL, d log L / dx.  `logdetP` is used by the dense kinds. */
static double orc_loglik_impl(const orc_lik_t *lk, double logdetP, const double *x, double *grad)
{
    const int d = lk->d;
    const double log2pi = 1.8378770664093454835606594728112;
    if (lk->kind == ORC_LIK_ROSEN) {
        /* log L = -scale * sum_{i=0}^{d-2} [100 (x_{i+1} - x_i^2)^2 + (1 - x_i)^2] */
        double s = 0.0;
        if (grad) for (int i = 0; i < d; ++i) grad[i] = 0.0;
        for (int i = 0; i + 1 < d; ++i) {
            double a = x[i + 1] - x[i] * x[i];
            double b = 1.0 - x[i];
            s += 100.0 * a * a + b * b;
            if (grad) {
                grad[i] += -lk->rosen_scale * (-400.0 * x[i] * a - 2.0 * b);
                grad[i + 1] += -lk->rosen_scale * (200.0 * a);
            }
        }
        return -lk->rosen_scale * s;
    }
    if (lk->kind == ORC_LIK_TORUS) {
        /* eq. torus: R = (sum over even i of sin(alpha x_i) + sum over odd j of
         * cos(beta x_j) + c)^3 with the paper's 1-based indices, i.e. sin on the
         * 0-based odd coordinates and cos on the 0-based even ones; log L = log R =
         * 3 log(S + c), defined while S + c > 0 (c > d keeps it so everywhere). */
        double s = lk->torus_c;
        for (int i = 0; i < d; ++i)
            s += (i & 1) ? sin(lk->torus_alpha * x[i]) : cos(lk->torus_beta * x[i]);
        if (!(s > 0.0)) {
            if (grad) for (int i = 0; i < d; ++i) grad[i] = 0.0;
            return -INFINITY;
        }
        if (grad)
            for (int i = 0; i < d; ++i)
                grad[i] = 3.0 / s * ((i & 1) ? lk->torus_alpha * cos(lk->torus_alpha * x[i])
                                              : -lk->torus_beta * sin(lk->torus_beta * x[i]));
        return 3.0 * log(s);
    }
    const int K = (lk->kind == ORC_LIK_ISO || lk->kind == ORC_LIK_DENSE) ? 1 : lk->n_comp;
    const int dense = (lk->kind == ORC_LIK_DENSE || lk->kind == ORC_LIK_DENSE_MIX);
    double *term = (double *)malloc(sizeof(double) * (size_t)K);
    double *r = (double *)malloc(sizeof(double) * (size_t)d);
    double *y = (double *)malloc(sizeof(double) * (size_t)d * (size_t)K);
    for (int k = 0; k < K; ++k) {
        const double *mu = lk->means + (size_t)k * d;
        for (int i = 0; i < d; ++i) r[i] = x[i] - mu[i];
        double q = 0.0;
        double *yk = y + (size_t)k * d;
        if (dense) {
            /* y = P (x - mu), q = (x - mu)^T P (x - mu) */
            for (int i = 0; i < d; ++i) {
                double t = 0.0;
                for (int j = 0; j < d; ++j) t += lk->precision[(size_t)i * d + j] * r[j];
                yk[i] = t;
                q += r[i] * t;
            }
            term[k] = (K > 1 ? orc_comp_logw(lk, k) : 0.0) - 0.5 * q;
        } else {
            double s2 = lk->sigma[k] * lk->sigma[k];
            for (int i = 0; i < d; ++i) { yk[i] = r[i] / s2; q += r[i] * r[i]; }
            term[k] = (K > 1 ? orc_comp_logw(lk, k) : 0.0) - 0.5 * q / s2 - 0.5 * d * (log2pi + log(s2));
        }
    }
    double m = term[0];
    for (int k = 1; k < K; ++k) if (term[k] > m) m = term[k];
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += exp(term[k] - m);
    double lse = (isfinite(m) ? m + log(s) : m);
    if (grad) {
        /* d log L / dx = - sum_k resp_k y_k, resp_k = exp(term_k - lse) */
        for (int i = 0; i < d; ++i) grad[i] = 0.0;
        for (int k = 0; k < K; ++k) {
            double resp = (K > 1) ? exp(term[k] - lse) : 1.0;
            for (int i = 0; i < d; ++i) grad[i] -= resp * y[(size_t)k * d + i];
        }
    }
    free(term); free(r); free(y);
    if (dense) lse += 0.5 * logdetP - 0.5 * d * log2pi;
    return lse;
}

/* Public wrapper (computes log det P on every call: test use only). */
double orc_loglik(const orc_lik_t *lk, const double *x, double *grad)
{
    double ld = 0.0;
    if (lk->kind == ORC_LIK_DENSE || lk->kind == ORC_LIK_DENSE_MIX) ld = orc_logdet_spd(lk->d, lk->precision);
    return orc_loglik_impl(lk, ld, x, grad);
}

/* d log L / d mu_k for k = 0..K-1 at x, written to dmu[K][d] (the parameter gradient
 * used by the posterior-weighted backward). */
void orc_loglik_dmeans(const orc_lik_t *lk, const double *x, double *dmu)
{
    const int d = lk->d;
    if (lk->kind == ORC_LIK_TORUS) {
        for (int i = 0; i < d; ++i) dmu[i] = 0.0; /* no component means */
        return;
    }
    const int K = (lk->kind == ORC_LIK_ISO || lk->kind == ORC_LIK_DENSE) ? 1 : lk->n_comp;
    const int dense = (lk->kind == ORC_LIK_DENSE || lk->kind == ORC_LIK_DENSE_MIX);
    const double log2pi = 1.8378770664093454835606594728112;
    double *term = (double *)malloc(sizeof(double) * (size_t)K);
    double *y = (double *)malloc(sizeof(double) * (size_t)d * (size_t)K);
    for (int k = 0; k < K; ++k) {
        const double *mu = lk->means + (size_t)k * d;
        double q = 0.0;
        double *yk = y + (size_t)k * d;
        if (dense) {
            for (int i = 0; i < d; ++i) {
                double t = 0.0;
                for (int j = 0; j < d; ++j) t += lk->precision[(size_t)i * d + j] * (x[j] - mu[j]);
                yk[i] = t;
                q += (x[i] - mu[i]) * t;
            }
            term[k] = (K > 1 ? orc_comp_logw(lk, k) : 0.0) - 0.5 * q;
        } else {
            double s2 = lk->sigma[k] * lk->sigma[k];
            for (int i = 0; i < d; ++i) { yk[i] = (x[i] - mu[i]) / s2; q += (x[i] - mu[i]) * (x[i] - mu[i]); }
            term[k] = (K > 1 ? orc_comp_logw(lk, k) : 0.0) - 0.5 * q / s2 - 0.5 * d * (log2pi + log(s2));
        }
    }
    double m = term[0];
    for (int k = 1; k < K; ++k) if (term[k] > m) m = term[k];
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += exp(term[k] - m);
    double lse = m + log(s);
    for (int k = 0; k < K; ++k) {
        double resp = (K > 1) ? exp(term[k] - lse) : 1.0;
        for (int i = 0; i < d; ++i) dmu[(size_t)k * d + i] = resp * y[(size_t)k * d + i];
    }
    free(term); free(y);
}

/* The reflection equation of Section 2.3: p' = p - 2 (p.n) n for a unit normal n. */
void orc_reflect(int d, double *p, const double *n)
{
    double pn = 0.0;
    for (int i = 0; i < d; ++i) pn += p[i] * n[i];
    for (int i = 0; i < d; ++i) p[i] = p[i] - 2.0 * pn * n[i];
}

/* ------------------------------------------------------------------------- */
/* One deterministic step of the walk (no noise, no prior box)                 */
/* ------------------------------------------------------------------------- */
/* mode 0 (Algorithm 5): x += p dt, then, if the new x is outside the slice
 * (log L <= L*), p is reflected with the normal n = grad log L / |grad log L|
 * taken at the new x.  mode 1 (the symmetric splitting): x += p dt / 2, the same
 * reflection test and normal at that half-step point, then x += p dt / 2.  The
 * second is time-reversible: applied to (x', -p') it returns (x, -p).  Returns 1 if
 * the step reflected.  Used by the reversibility pins. */
int orc_walk_step(const orc_lik_t *lk, double logdetP, int mode, double lstar, double dt, double *x, double *p)
{
    const int d = lk->d;
    double *g = (double *)malloc(sizeof(double) * d);
    const double h = mode ? 0.5 * dt : dt;
    for (int i = 0; i < d; ++i) x[i] += p[i] * h;
    const double logl = orc_loglik_impl(lk, logdetP, x, g);
    int refl = 0;
    if (!(logl > lstar)) {
        double gg = 0.0;
        for (int i = 0; i < d; ++i) gg += g[i] * g[i];
        const double gn = sqrt(gg);
        if (gn > 0.0 && isfinite(gn)) {
            for (int i = 0; i < d; ++i) g[i] /= gn;
            orc_reflect(d, p, g);
        } else {
            for (int i = 0; i < d; ++i) p[i] = -p[i];
        }
        refl = 1;
    }
    if (mode)
        for (int i = 0; i < d; ++i) x[i] += p[i] * h;
    free(g);
    return refl;
}

/* ------------------------------------------------------------------------- */
/* Batched Hamiltonian slice sampling (Algorithm 5)                           */
/* ------------------------------------------------------------------------- */

typedef struct {
    int n_live, n_steps, min_steps;
    double dt_init, delta_p, tol;
    int min_ref, max_ref, prune_after, termination, clustering;
    uint64_t seed;
    uint32_t run_id;
    int max_iters;
    int noise_mode;
    double out_lo, out_hi;
    int periodic; /* 1: the prior box is a torus, positions wrap instead of reflecting */
    int keep_last; /* 1: return the last saved state instead of a uniform one (App. G ablation) */
    int noise_inside; /* 1: the momentum noise perturbs inside steps only; an outside step only reflects */
    int pick_all;     /* 1: the pick is uniform over every step of the saving window and an outside
                         step returns the start point (rejection); 0: uniform over saved inside states */
    int territory;    /* 1: with several clusters alive, a new point whose nearest surviving point
                         belongs to another cluster is rejected (the walker returns its start point) */
    int box_fold;     /* 1: the prior box reflects a walker exactly (the position folds back across
                         the face and the momentum component flips; not an outside step); 0: leaving
                         the box is an outside step that reflects off the violated faces */
    int fold_counts;  /* with box_fold: an inside step on which the box reflected the walker counts
                         as a reflection for the step-size control (not for n_ref or the pick) */
    int midpoint;     /* 1: the time-reversible form of the step (an option, not the default):
                         half move, reflection with the normal at the half step if that point is
                         outside, half move; the states (saved, picked) are the whole-step points,
                         the refresh noise acts on every state, and the picked state is tested
                         against L* at the end (outside: the walker returns its start point) */
} orc_cfg_t;

typedef struct {
    long n_in, n_out;     /* inside / outside steps over all walkers          */
    int t_save, t_stop;   /* first saving step, last step taken               */
    int n_fallback;       /* walkers that saved nothing and return their start */
    long n_fold;          /* inside steps on which the box reflected the walker (box_fold) */
} orc_batch_stats_t;

/*
 * Evolve n walkers together from x0[n][d] (all inside the slice L > lstar) with
 * step dt, as Algorithm 5 states it for the whole batch:
 *   - p ~ N(0, I) per walker;
 *   - every step, every walker: x += p dt; evaluate log L and its gradient;
 *     outside = not (L > L*) or outside the prior box; outside walkers reflect
 *     p -= 2 (p.n) n with n the unit score (or the outward box normal); every
 *     momentum takes the noise (noise_mode 0: p *= 1 + delta_p eps, as
 *     printed in Algorithm 5; noise_mode 1: p = sqrt(1-delta_p^2) p + delta_p
 *     eps, the noise "added" of Section 3 in the form that keeps p ~ N(0, I));
 *     n_ref += outside;
 *   - inside states are saved once min over walkers of n_ref >= min_ref (the
 *     text's "after a designated number of reflections");
 *   - the loop runs while min over walkers of n_ref < max_ref (and at least
 *     min_steps, at most n_steps steps).
 * Each walker returns one state drawn uniformly from its own saved inside states
 * (a size-1 reservoir; replacement with probability 1/count), or its start point
 * if it saved none.  With pick_all the reservoir runs over every step of the
 * saving window, inside or outside, and a drawn outside step is a rejection: the
 * walker returns its start point.  With noise_inside an outside step reflects
 * and takes no noise.  Walkers that stay outside for prune_after consecutive steps
 * are reset to their start point with a fresh momentum (Section 3, pruning).
 * Random numbers: walker j uses slot j of iteration `iter`.
 * If trace != NULL it receives, per step t and walker j, x then p then logL and
 * the outside flag: trace[((t-1)*n + j)*(2d+2) + ...], for t <= n_steps.
 */
/* The prior box as an exact reflection on a position (box_fold): the path unfolded on
 * a line of period 2w folds back; an odd number of crossings flips p_i. */
static int fold_into_box(int d, const double *lo, const double *hi, double *xj, double *pj)
{
    int folded = 0;
    for (int i = 0; i < d; ++i) {
        if (xj[i] >= lo[i] && xj[i] <= hi[i]) continue;
        folded = 1;
        const double w = hi[i] - lo[i];
        double u = fmod(xj[i] - lo[i], 2.0 * w);
        if (u < 0.0) u += 2.0 * w;
        if (u > w) { xj[i] = lo[i] + (2.0 * w - u); pj[i] = -pj[i]; }
        else xj[i] = lo[i] + u;
    }
    return folded;
}

/* Algorithm 5 with the time-reversible step (cfg->midpoint; see orc_walk_step mode 1):
 * the walker's state m moves half a step to z, where log L and its gradient are
 * evaluated (the reflection test, n_ref, the outside fraction), reflects there if z is
 * outside, moves the second half step, and takes the refresh noise
 * p <- sqrt(1 - dp^2) p + dp eps.  The prior box reflects exactly on both half moves.
 * The saving window, the global stop and the size-1 reservoir are those of
 * orc_hss_batch, over every step's state m; the drawn state is tested against L* at
 * the end and, outside, the walker returns its start point (trace rows hold m, p, the
 * log L at z and the outside flag of z).  keep_last (the App. G fixed-step ablation)
 * keeps the last state of the window in place of the reservoir's draw; with a fixed
 * number of steps (max_ref out of reach, min_ref 0, no pruning) the walk is then a
 * fixed-length reversible trajectory whose end point is accepted when inside. */
static int hss_batch_mid(const orc_lik_t *lk, double logdetP, const double *lo, const double *hi,
                         const orc_cfg_t *cfg, uint32_t iter, int n, const double *x0, const double *logl0,
                         double lstar, double dt, double *x_out, double *logl_out, int *steps_out,
                         orc_batch_stats_t *st, double *trace)
{
    const int d = lk->d;
    const size_t nd = (size_t)n * d;
    double *m = (double *)malloc(sizeof(double) * nd);
    double *p = (double *)malloc(sizeof(double) * nd);
    double *xr = (double *)malloc(sizeof(double) * nd);
    double *z = (double *)malloc(sizeof(double) * d);
    double *g = (double *)malloc(sizeof(double) * d);
    double *eps = (double *)malloc(sizeof(double) * d);
    int *n_ref = (int *)calloc(n, sizeof(int));
    int *consec = (int *)calloc(n, sizeof(int));
    int *count = (int *)calloc(n, sizeof(int));
    long n_in = 0, n_out = 0, n_fold = 0;
    int t_save = 0, t = 0, saving = 0;
    memcpy(m, x0, sizeof(double) * nd);
    for (int j = 0; j < n; ++j)
        orc_normals(cfg->seed, cfg->run_id, iter, ORC_P_MOM, (uint32_t)j, 0, d, p + (size_t)j * d);
    const double keep = sqrt(1.0 - cfg->delta_p * cfg->delta_p);
    for (;;) {
        int min_ref_now = n_ref[0];
        for (int j = 1; j < n; ++j) if (n_ref[j] < min_ref_now) min_ref_now = n_ref[j];
        if (n == 0 || t >= cfg->n_steps) break;
        if (min_ref_now >= cfg->max_ref && t >= cfg->min_steps) break;
        ++t;
        for (int j = 0; j < n; ++j) {
            double *mj = m + (size_t)j * d, *pj = p + (size_t)j * d;
            for (int i = 0; i < d; ++i) z[i] = mj[i] + 0.5 * pj[i] * dt;
            int folded = fold_into_box(d, lo, hi, z, pj);
            const double logl = orc_loglik_impl(lk, logdetP, z, g);
            const int out = !(logl > lstar);
            if (out) {
                double gg = 0.0;
                for (int i = 0; i < d; ++i) gg += g[i] * g[i];
                const double gn = sqrt(gg);
                if (gn > 0.0 && isfinite(gn)) {
                    for (int i = 0; i < d; ++i) g[i] /= gn;
                    orc_reflect(d, pj, g);
                } else {
                    for (int i = 0; i < d; ++i) pj[i] = -pj[i];
                }
            }
            for (int i = 0; i < d; ++i) mj[i] = z[i] + 0.5 * pj[i] * dt;
            folded |= fold_into_box(d, lo, hi, mj, pj);
            orc_normals(cfg->seed, cfg->run_id, iter, ORC_P_NOISE, (uint32_t)j, (uint32_t)t, d, eps);
            for (int i = 0; i < d; ++i) pj[i] = keep * pj[i] + cfg->delta_p * eps[i];
            if (trace) {
                double *tr = trace + ((size_t)(t - 1) * n + j) * (2 * d + 2);
                for (int i = 0; i < d; ++i) { tr[i] = mj[i]; tr[d + i] = pj[i]; }
                tr[2 * d] = logl; tr[2 * d + 1] = out;
            }
            n_ref[j] += out;
            if (out) { ++n_out; ++consec[j]; } else { ++n_in; consec[j] = 0; n_fold += folded; }
        }
        if (!saving) {
            int mr = n_ref[0];
            for (int j = 1; j < n; ++j) if (n_ref[j] < mr) mr = n_ref[j];
            if (mr >= cfg->min_ref) { saving = 1; t_save = t; }
        }
        for (int j = 0; j < n; ++j) {
            if (saving) {
                ++count[j];
                uint32_t w[4];
                orc_rng_block(cfg->seed, cfg->run_id, iter, ORC_P_NOISE, (uint32_t)j, (uint32_t)t, 0, w);
                uint32_t word = (w[0] & 511u) | ((w[1] & 511u) << 9) | ((w[2] & 511u) << 18) | ((w[3] & 31u) << 27);
                if (cfg->keep_last || (((uint64_t)word * (uint64_t)count[j]) >> 32) == 0)
                    memcpy(xr + (size_t)j * d, m + (size_t)j * d, sizeof(double) * d);
            }
            if (cfg->prune_after > 0 && consec[j] >= cfg->prune_after) {
                memcpy(m + (size_t)j * d, x0 + (size_t)j * d, sizeof(double) * d);
                orc_normals(cfg->seed, cfg->run_id, iter, ORC_P_PRUNE, (uint32_t)j, (uint32_t)t, d,
                            p + (size_t)j * d);
                consec[j] = 0;
            }
        }
    }
    int n_fb = 0;
    for (int j = 0; j < n; ++j) {
        double l = -INFINITY;
        if (count[j] > 0) l = orc_loglik_impl(lk, logdetP, xr + (size_t)j * d, g);
        if (count[j] > 0 && l > lstar) {
            memcpy(x_out + (size_t)j * d, xr + (size_t)j * d, sizeof(double) * d);
            logl_out[j] = l;
        } else {
            memcpy(x_out + (size_t)j * d, x0 + (size_t)j * d, sizeof(double) * d);
            logl_out[j] = logl0[j];
            ++n_fb;
        }
        if (steps_out) steps_out[j] = t;
    }
    if (st) {
        st->n_in = n_in; st->n_out = n_out; st->t_save = t_save; st->t_stop = t; st->n_fallback = n_fb;
        st->n_fold = n_fold;
    }
    free(m); free(p); free(xr); free(z); free(g); free(eps);
    free(n_ref); free(consec); free(count);
    return 0;
}

int orc_hss_batch(const orc_lik_t *lk, double logdetP, const double *lo, const double *hi,
                  const orc_cfg_t *cfg, uint32_t iter, int n, const double *x0, const double *logl0,
                  double lstar, double dt, double *x_out, double *logl_out, int *steps_out,
                  orc_batch_stats_t *st, double *trace)
{
    if (cfg->midpoint && !cfg->periodic)
        return hss_batch_mid(lk, logdetP, lo, hi, cfg, iter, n, x0, logl0, lstar, dt, x_out, logl_out, steps_out, st,
                             trace);
    const int d = lk->d;
    const size_t nd = (size_t)n * d;
    double *x = (double *)malloc(sizeof(double) * nd);
    double *p = (double *)malloc(sizeof(double) * nd);
    double *xr = (double *)malloc(sizeof(double) * nd);
    double *lr = (double *)malloc(sizeof(double) * n);
    double *g = (double *)malloc(sizeof(double) * d);
    double *nrm = (double *)malloc(sizeof(double) * d);
    double *eps = (double *)malloc(sizeof(double) * d);
    int *n_ref = (int *)calloc(n, sizeof(int));
    int *consec = (int *)calloc(n, sizeof(int));
    int *count = (int *)calloc(n, sizeof(int));
    int *outside = (int *)calloc(n, sizeof(int));
    double *logl_now = (double *)malloc(sizeof(double) * n);
    long n_in = 0, n_out = 0, n_fold = 0;
    int t_save = 0, t = 0, saving = 0;
    memcpy(x, x0, sizeof(double) * nd);
    for (int j = 0; j < n; ++j)
        orc_normals(cfg->seed, cfg->run_id, iter, ORC_P_MOM, (uint32_t)j, 0, d, p + (size_t)j * d);
    for (;;) {
        /* loop condition: min over walkers of n_ref < max_ref, or fewer than
         * min_steps steps taken; never more than n_steps steps */
        int min_ref_now = n_ref[0];
        for (int j = 1; j < n; ++j) if (n_ref[j] < min_ref_now) min_ref_now = n_ref[j];
        if (n == 0 || t >= cfg->n_steps) break;
        if (min_ref_now >= cfg->max_ref && t >= cfg->min_steps) break;
        ++t;
        for (int j = 0; j < n; ++j) {
            double *xj = x + (size_t)j * d, *pj = p + (size_t)j * d;
            /* x += p dt; on a periodic prior the position wraps into [lo, hi) */
            for (int i = 0; i < d; ++i) xj[i] = xj[i] + pj[i] * dt;
            if (cfg->periodic)
                for (int i = 0; i < d; ++i) {
                    const double w = hi[i] - lo[i];
                    double u = fmod(xj[i] - lo[i], w);
                    if (u < 0.0) u += w;
                    xj[i] = lo[i] + u;
                }
            int folded = 0;
            if (!cfg->periodic && cfg->box_fold)
                for (int i = 0; i < d; ++i) {
                    /* specular reflection off the faces lo_i, hi_i: the path unfolded on a
                     * line of period 2w folds back; an odd number of crossings flips p_i */
                    if (xj[i] >= lo[i] && xj[i] <= hi[i]) continue;
                    folded = 1;
                    const double w = hi[i] - lo[i];
                    double u = fmod(xj[i] - lo[i], 2.0 * w);
                    if (u < 0.0) u += 2.0 * w;
                    if (u > w) { xj[i] = lo[i] + (2.0 * w - u); pj[i] = -pj[i]; }
                    else xj[i] = lo[i] + u;
                }
            /* one fused evaluation of log L and its gradient */
            double logl = orc_loglik_impl(lk, logdetP, xj, g);
            int inbox = 1;
            for (int i = 0; i < d; ++i) if (!(xj[i] >= lo[i] && xj[i] <= hi[i])) inbox = 0;
            int out = (!inbox) || !(logl > lstar);
            if (out) {
                int have_n = 1;
                if (!inbox) {
                    /* outward normal of the violated prior-box faces */
                    double nn = 0.0;
                    for (int i = 0; i < d; ++i) {
                        nrm[i] = (xj[i] < lo[i]) ? -1.0 : (xj[i] > hi[i] ? 1.0 : 0.0);
                        nn += nrm[i] * nrm[i];
                    }
                    nn = sqrt(nn);
                    for (int i = 0; i < d; ++i) nrm[i] /= nn;
                } else {
                    /* n = grad log L / |grad log L| (reflection equation) */
                    double gg = 0.0;
                    for (int i = 0; i < d; ++i) gg += g[i] * g[i];
                    double gn = sqrt(gg);
                    if (gn > 0.0 && isfinite(gn)) {
                        for (int i = 0; i < d; ++i) nrm[i] = g[i] / gn;
                    } else {
                        have_n = 0; /* no usable normal: reverse the momentum */
                        for (int i = 0; i < d; ++i) pj[i] = -pj[i];
                    }
                }
                if (have_n) orc_reflect(d, pj, nrm);
            }
            /* momentum noise, eps ~ N(0, I) fresh every step and walker:
             *   noise_mode 0: p <- p (1 + delta_p eps)            (Algorithm 5 as printed)
             *   noise_mode 1: p <- sqrt(1 - delta_p^2) p + delta_p eps
             *                 (noise added, Section 3, in the form that keeps p ~ N(0, I)) */
            orc_normals(cfg->seed, cfg->run_id, iter, ORC_P_NOISE, (uint32_t)j, (uint32_t)t, d, eps);
            if (cfg->noise_inside && out) {
                /* an outside step only reflects */
            } else if (cfg->noise_mode == 1) {
                double keep = sqrt(1.0 - cfg->delta_p * cfg->delta_p);
                for (int i = 0; i < d; ++i) pj[i] = keep * pj[i] + cfg->delta_p * eps[i];
            } else {
                for (int i = 0; i < d; ++i) pj[i] = pj[i] * (1.0 + cfg->delta_p * eps[i]);
            }
            if (trace) {
                double *tr = trace + ((size_t)(t - 1) * n + j) * (2 * d + 2);
                for (int i = 0; i < d; ++i) { tr[i] = xj[i]; tr[d + i] = pj[i]; }
                tr[2 * d] = logl; tr[2 * d + 1] = out;
            }
            n_ref[j] += out;
            outside[j] = out;
            logl_now[j] = logl;
            if (out) { ++n_out; ++consec[j]; } else { ++n_in; consec[j] = 0; n_fold += folded; }
        }
        /* trajectory preservation: save inside states once every walker has
         * reflected at least min_ref times */
        if (!saving) {
            int mr = n_ref[0];
            for (int j = 1; j < n; ++j) if (n_ref[j] < mr) mr = n_ref[j];
            if (mr >= cfg->min_ref) { saving = 1; t_save = t; }
        }
        for (int j = 0; j < n; ++j) {
            if (saving && (!outside[j] || cfg->pick_all)) {
                ++count[j];
                /* acceptance word: the low bits of the four words of noise block 0
                 * of this step, which the uniforms (top 23 bits) leave unused */
                uint32_t w[4];
                orc_rng_block(cfg->seed, cfg->run_id, iter, ORC_P_NOISE, (uint32_t)j, (uint32_t)t, 0, w);
                uint32_t word = (w[0] & 511u) | ((w[1] & 511u) << 9) | ((w[2] & 511u) << 18) | ((w[3] & 31u) << 27);
                /* keep_last: the App. G ablation that integrates a fixed number of steps and
                 * keeps the last sample, in place of the size-1 reservoir */
                if (cfg->keep_last || (((uint64_t)word * (uint64_t)count[j]) >> 32) == 0) {
                    if (outside[j]) { /* rejection: the walker keeps its start point */
                        memcpy(xr + (size_t)j * d, x0 + (size_t)j * d, sizeof(double) * d);
                        lr[j] = logl0[j];
                    } else {
                        memcpy(xr + (size_t)j * d, x + (size_t)j * d, sizeof(double) * d);
                        lr[j] = logl_now[j];
                    }
                }
            }
            if (cfg->prune_after > 0 && consec[j] >= cfg->prune_after) {
                /* pruning: back to the start point with a fresh momentum */
                memcpy(x + (size_t)j * d, x0 + (size_t)j * d, sizeof(double) * d);
                orc_normals(cfg->seed, cfg->run_id, iter, ORC_P_PRUNE, (uint32_t)j, (uint32_t)t, d,
                            p + (size_t)j * d);
                consec[j] = 0;
            }
        }
    }
    int n_fb = 0;
    for (int j = 0; j < n; ++j) {
        if (count[j] > 0) {
            memcpy(x_out + (size_t)j * d, xr + (size_t)j * d, sizeof(double) * d);
            logl_out[j] = lr[j];
        } else {
            memcpy(x_out + (size_t)j * d, x0 + (size_t)j * d, sizeof(double) * d);
            logl_out[j] = logl0[j];
            ++n_fb;
        }
        if (steps_out) steps_out[j] = t;
    }
    if (st) {
        st->n_in = n_in; st->n_out = n_out; st->t_save = t_save; st->t_stop = t; st->n_fallback = n_fb;
        st->n_fold = n_fold;
    }
    free(x); free(p); free(xr); free(lr); free(g); free(nrm); free(eps);
    free(n_ref); free(consec); free(count); free(outside); free(logl_now);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Ordering: ascending (log L, slot); NaN counts as the lowest                */
/* ------------------------------------------------------------------------- */

static _Thread_local const double *g_sort_key; /* per thread: runs may execute concurrently */
static int orc_cmp_key(const void *a, const void *b)
{
    int i = *(const int *)a, j = *(const int *)b;
    double x = g_sort_key[i], y = g_sort_key[j];
    int xn = isnan(x), yn = isnan(y);
    if (xn != yn) return xn ? -1 : 1;
    if (!xn) { if (x < y) return -1; if (x > y) return 1; }
    return (i < j) ? -1 : (i > j ? 1 : 0);
}

/* order[0..n) = slots sorted ascending by (logl, slot). */
void orc_sort_by_logl(int n, const double *logl, int *order)
{
    for (int i = 0; i < n; ++i) order[i] = i;
    g_sort_key = logl;
    qsort(order, (size_t)n, sizeof(int), orc_cmp_key);
}

/* ------------------------------------------------------------------------- */
/* Cluster finding (Algorithm 4): k-NN graph components                       */
/* ------------------------------------------------------------------------- */

static int uf_find(int *par, int i)
{
    while (par[i] != i) i = par[i];
    return i;
}

/* Union by smallest root; returns 1 if two components were merged. */
static int uf_union(int *par, int a, int b)
{
    int ra = uf_find(par, a), rb = uf_find(par, b);
    if (ra == rb) return 0;
    if (ra < rb) par[rb] = ra; else par[ra] = rb;
    return 1;
}

typedef struct { float dist; int idx; } orc_nb_t;
static int orc_cmp_nb(const void *a, const void *b)
{
    const orc_nb_t *u = (const orc_nb_t *)a, *v = (const orc_nb_t *)b;
    if (u->dist < v->dist) return -1;
    if (u->dist > v->dist) return 1;
    return (u->idx < v->idx) ? -1 : (u->idx > v->idx ? 1 : 0);
}

/*
 * Algorithm 4 on m points x[m][d] (FP32, the precision the decision is taken in;
 * squared distances accumulate in coordinate order, one fmaf per coordinate):
 * for k = 2, 3, ... build the k-nearest-neighbour graph (edge i-j when j is among
 * the k nearest of i, or i among the k nearest of j; Euclidean; ties broken by the
 * lower index; self excluded; k capped at m-1), take its connected components, and
 * stop at the first k whose component-size multiset equals that of k-1.  Because
 * the graph for k contains the graph for k-1, the multisets are equal exactly when
 * rank k merges no components.  Writes comp[i] = smallest member index of i's
 * component and returns the number of components.
 */
int orc_knn_components(int m, int d, const float *x, int *comp)
{
    if (m <= 0) return 0;
    int *par = (int *)malloc(sizeof(int) * m);
    for (int i = 0; i < m; ++i) par[i] = i;
    if (m >= 3) {
        int kmax = m - 1;
        orc_nb_t *nb = (orc_nb_t *)malloc(sizeof(orc_nb_t) * (size_t)m * kmax);
        orc_nb_t *row = (orc_nb_t *)malloc(sizeof(orc_nb_t) * m);
        for (int i = 0; i < m; ++i) {
            int c = 0;
            for (int j = 0; j < m; ++j) {
                if (j == i) continue;
                float s = 0.0f;
                for (int t = 0; t < d; ++t) {
                    float diff = x[(size_t)i * d + t] - x[(size_t)j * d + t];
                    s = fmaf(diff, diff, s); /* one correctly rounded fused multiply-add per coordinate */
                }
                row[c].dist = s; row[c].idx = j; ++c;
            }
            qsort(row, (size_t)c, sizeof(orc_nb_t), orc_cmp_nb);
            memcpy(nb + (size_t)i * kmax, row, sizeof(orc_nb_t) * kmax);
        }
        /* k = 2: ranks 1 and 2 */
        for (int i = 0; i < m; ++i) {
            uf_union(par, i, nb[(size_t)i * kmax + 0].idx);
            if (kmax >= 2) uf_union(par, i, nb[(size_t)i * kmax + 1].idx);
        }
        for (int k = 3; k <= kmax; ++k) {
            int merged = 0;
            for (int i = 0; i < m; ++i) merged += uf_union(par, i, nb[(size_t)i * kmax + (k - 1)].idx);
            if (!merged) break; /* sizes(k) == sizes(k-1) */
        }
        free(nb); free(row);
    }
    int ncomp = 0;
    for (int i = 0; i < m; ++i) {
        comp[i] = uf_find(par, i);
        if (comp[i] == i) ++ncomp;
    }
    free(par);
    return ncomp;
}

/* ------------------------------------------------------------------------- */
/* Summary statistics of Appendix H, in log space                             */
/* ------------------------------------------------------------------------- */

static double lae(double a, double b)
{
    if (a == ORC_NEG_INF) return b;
    if (b == ORC_NEG_INF) return a;
    double m = a > b ? a : b;
    return m + log1p(exp(-fabs(a - b)));
}
static double lae3(double a, double b, double c) { return lae(lae(a, b), c); }

typedef struct {
    int cap;              /* cluster slots                            */
    int *alive;           /* [cap]                                    */
    int *n;               /* [cap] live points per cluster            */
    double logZ, logZ2;   /* log Zbar, log Z^2bar                     */
    double *logZp, *logZp2, *logZXp, *logZpXp, *logXp, *logXp2; /* [cap] */
    double *logXX;        /* [cap][cap], symmetric, off-diagonal      */
} orc_stats_t;

static void stats_alloc(orc_stats_t *s, int cap)
{
    s->cap = cap;
    s->alive = (int *)calloc(cap, sizeof(int));
    s->n = (int *)calloc(cap, sizeof(int));
    s->logZp = (double *)malloc(sizeof(double) * cap);
    s->logZp2 = (double *)malloc(sizeof(double) * cap);
    s->logZXp = (double *)malloc(sizeof(double) * cap);
    s->logZpXp = (double *)malloc(sizeof(double) * cap);
    s->logXp = (double *)malloc(sizeof(double) * cap);
    s->logXp2 = (double *)malloc(sizeof(double) * cap);
    s->logXX = (double *)malloc(sizeof(double) * (size_t)cap * cap);
    for (int i = 0; i < cap; ++i) {
        s->logZp[i] = s->logZp2[i] = s->logZXp[i] = s->logZpXp[i] = ORC_NEG_INF;
        s->logXp[i] = s->logXp2[i] = ORC_NEG_INF;
    }
    for (size_t i = 0; i < (size_t)cap * cap; ++i) s->logXX[i] = ORC_NEG_INF;
    /* eqs. ini0-ini11: one cluster, Zbar = Z^2bar = ZXbar = 0, Xbar = X^2bar = 1 */
    s->logZ = ORC_NEG_INF;
    s->logZ2 = ORC_NEG_INF;
    s->alive[0] = 1;
    s->logXp[0] = 0.0;
    s->logXp2[0] = 0.0;
}

static void stats_free(orc_stats_t *s)
{
    free(s->alive); free(s->n); free(s->logZp); free(s->logZp2); free(s->logZXp);
    free(s->logZpXp); free(s->logXp); free(s->logXp2); free(s->logXX);
}

/*
 * Kill one point of log-likelihood L from cluster p: eqs. update0-update9 with
 * n_p the live count of p before the kill, all right-hand sides taken before the
 * update.  Returns log of the prior mass assigned to the dead point,
 * log(Xbar_p / (n_p + 1)).  Removes p when its count reaches zero (Algorithm 3).
 */
static double stats_kill(orc_stats_t *s, int p, double L)
{
    const double n = (double)s->n[p];
    const double ln2 = 0.69314718055994530941723212145818;
    const double a = log(n) - log(n + 1.0);     /* log n/(n+1)           */
    const double i1 = -log(n + 1.0);             /* log 1/(n+1)           */
    const double i2 = -log(n + 1.0) - log(n + 2.0); /* log 1/((n+1)(n+2)) */
    const double Xp = s->logXp[p], Xp2 = s->logXp2[p], ZXp = s->logZXp[p], ZpXp = s->logZpXp[p];
    const double logw = Xp + i1;
    /* update0, update1 */
    s->logZ = lae(s->logZ, Xp + L + i1);
    s->logZp[p] = lae(s->logZp[p], Xp + L + i1);
    /* update3, update4 */
    s->logZ2 = lae3(s->logZ2, ln2 + ZXp + L + i1, ln2 + Xp2 + 2.0 * L + i2);
    s->logZp2[p] = lae3(s->logZp2[p], ln2 + ZpXp + L + i1, ln2 + Xp2 + 2.0 * L + i2);
    /* update5, update7 */
    s->logZXp[p] = lae(ZXp + a, log(n) + Xp2 + L + i2);
    s->logZpXp[p] = lae(ZpXp + a, log(n) + Xp2 + L + i2);
    /* update6 and update9 for every other live cluster q */
    for (int q = 0; q < s->cap; ++q) {
        if (q == p || !s->alive[q]) continue;
        double XXpq = s->logXX[(size_t)p * s->cap + q];
        s->logZXp[q] = lae(s->logZXp[q], XXpq + L + i1);
        s->logXX[(size_t)p * s->cap + q] = XXpq + a;
        s->logXX[(size_t)q * s->cap + p] = XXpq + a;
    }
    /* update2, update8 */
    s->logXp[p] = Xp + a;
    s->logXp2[p] = Xp2 + log(n) - log(n + 2.0);
    s->n[p] -= 1;
    if (s->n[p] == 0) {
        s->alive[p] = 0;
        s->logZp[p] = s->logZp2[p] = s->logZXp[p] = s->logZpXp[p] = ORC_NEG_INF;
        s->logXp[p] = s->logXp2[p] = ORC_NEG_INF;
        for (int q = 0; q < s->cap; ++q) {
            s->logXX[(size_t)p * s->cap + q] = ORC_NEG_INF;
            s->logXX[(size_t)q * s->cap + p] = ORC_NEG_INF;
        }
    }
    return logw;
}

/*
 * Split cluster p (n points) into parts with sizes sz[0..np), part 0 keeping id p
 * and part i > 0 taking id ids[i]: eqs. new0-new6, with new3 applied to
 * Y in {Z, X_q} for every other live cluster q.
 */
static void stats_split(orc_stats_t *s, int p, int np, const int *sz, const int *ids)
{
    const double n = (double)s->n[p];
    const double Xp = s->logXp[p], Xp2 = s->logXp2[p], Zp = s->logZp[p], Zp2 = s->logZp2[p];
    const double ZXp = s->logZXp[p], ZpXp = s->logZpXp[p];
    double *XXold = (double *)malloc(sizeof(double) * s->cap);
    for (int q = 0; q < s->cap; ++q) XXold[q] = s->logXX[(size_t)p * s->cap + q];
    int *others = (int *)calloc(s->cap, sizeof(int));
    for (int q = 0; q < s->cap; ++q) others[q] = (s->alive[q] && q != p);
    for (int i = 0; i < np; ++i) {
        int c = ids[i];
        double ni = (double)sz[i];
        double fi = log(ni) - log(n);                                  /* n_i / n               */
        double gi = log(ni) + log(ni + 1.0) - log(n) - log(n + 1.0);   /* n_i(n_i+1)/(n(n+1))   */
        s->alive[c] = 1;
        s->n[c] = sz[i];
        s->logXp[c] = fi + Xp;       /* new0 */
        s->logXp2[c] = gi + Xp2;     /* new1 */
        s->logZXp[c] = fi + ZXp;     /* new3, Y = Z */
        s->logZp[c] = fi + Zp;       /* new4 */
        s->logZpXp[c] = gi + ZpXp;   /* new5 */
        s->logZp2[c] = gi + Zp2;     /* new6 */
    }
    for (int i = 0; i < np; ++i) {
        int c = ids[i];
        double fi = log((double)sz[i]) - log(n);
        for (int q = 0; q < s->cap; ++q) {
            if (!others[q]) continue;
            /* new3, Y = X_q */
            s->logXX[(size_t)c * s->cap + q] = fi + XXold[q];
            s->logXX[(size_t)q * s->cap + c] = fi + XXold[q];
        }
        for (int j = 0; j < np; ++j) {
            if (j == i) continue;
            /* new2 */
            double v = log((double)sz[i]) + log((double)sz[j]) - log(n) - log(n + 1.0) + Xp2;
            s->logXX[(size_t)c * s->cap + ids[j]] = v;
        }
    }
    free(XXold); free(others);
}

/* Exported for component tests: run update0-update9 on a kill sequence, starting
 * from one cluster per distinct label with the given counts and log X (other
 * statistics zero).  Outputs the final log Z, log Z^2, per-cluster log X and the
 * log mass of every kill. */
void orc_stats_sequence(int n_clusters, const int *counts, const double *logX0,
                        const double *logZX0, const double *logXX0,
                        int k, const int *labels, const double *logl,
                        double *out_logZ, double *out_logZ2, double *out_logX,
                        double *out_logX2, double *out_logZX, double *out_logw)
{
    orc_stats_t s;
    stats_alloc(&s, n_clusters);
    for (int c = 0; c < n_clusters; ++c) {
        s.alive[c] = counts[c] > 0;
        s.n[c] = counts[c];
        s.logXp[c] = logX0[c];
        s.logXp2[c] = 2.0 * logX0[c];
        s.logZXp[c] = logZX0 ? logZX0[c] : ORC_NEG_INF;
        for (int q = 0; q < n_clusters; ++q)
            s.logXX[(size_t)c * n_clusters + q] = (logXX0 && q != c) ? logXX0[(size_t)c * n_clusters + q] : ORC_NEG_INF;
    }
    for (int i = 0; i < k; ++i) out_logw[i] = stats_kill(&s, labels[i], logl[i]);
    *out_logZ = s.logZ;
    *out_logZ2 = s.logZ2;
    for (int c = 0; c < n_clusters; ++c) {
        out_logX[c] = s.logXp[c];
        if (out_logX2) out_logX2[c] = s.logXp2[c];
        if (out_logZX) out_logZX[c] = s.logZXp[c];
    }
    stats_free(&s);
}

/* Exported for tests: a small program of kills and two-way splits applied to
 * the statistics, starting from one cluster (id 0) of n0 live points with
 * X = 1 (eqs. ini0-ini11).  op[i] = 0: kill a point of log-likelihood val[i]
 * from cluster arg[i] (update0-update9).  op[i] = 1: split cluster arg[i] into a
 * part of (int)val[i] points keeping the id and a part with the remaining points
 * taking the lowest free id (new0-new6).  out receives logZ, logZ2 and then, for
 * each of the `cap` cluster slots: logXp, logXp2, logZXp, logZp, logZp2,
 * logZpXp, n_p; followed by the cap*cap matrix logXX. */
void orc_stats_program(int cap, int n0, int n_ops, const int *op, const int *arg, const double *val,
                       double *out)
{
    orc_stats_t st;
    stats_alloc(&st, cap);
    st.n[0] = n0;
    for (int i = 0; i < n_ops; ++i) {
        if (op[i] == 0) {
            stats_kill(&st, arg[i], val[i]);
        } else {
            int p = arg[i];
            int sz[2] = {(int)val[i], st.n[p] - (int)val[i]};
            int ids[2] = {p, 0};
            while (st.alive[ids[1]] || ids[1] == p) ++ids[1];
            stats_split(&st, p, 2, sz, ids);
        }
    }
    out[0] = st.logZ;
    out[1] = st.logZ2;
    for (int c = 0; c < cap; ++c) {
        double *o = out + 2 + 7 * c;
        o[0] = st.logXp[c]; o[1] = st.logXp2[c]; o[2] = st.logZXp[c]; o[3] = st.logZp[c];
        o[4] = st.logZp2[c]; o[5] = st.logZpXp[c]; o[6] = st.n[c];
    }
    for (int i = 0; i < cap * cap; ++i) out[2 + 7 * cap + i] = st.logXX[i];
    stats_free(&st);
}

/* ------------------------------------------------------------------------- */
/* Cluster regions of the new points                                          */
/* ------------------------------------------------------------------------- */

/*
 * The cluster statistics of Appendix H hold when the live points of cluster p are
 * spread over p's own region only.  A walker spawned in cluster p (Algorithm 3:
 * the cluster is chosen with probability Xbar_p / sum Xbar, the start point among
 * p's survivors) can cross into the region of another cluster while the two are
 * still connected; kept with label p, it would add points to a region whose volume
 * another cluster accounts for.  So the new point j is kept only if its nearest
 * surviving point (FP32 squared distances accumulated in coordinate order, one
 * fmaf per coordinate, ties to the lower index; the precision the cluster finding
 * decides in) carries the label it was spawned with; otherwise it is rejected and
 * the walker returns its start point.
 * surv[m_s][d] FP32, surv_label[m_s]; xn[k][d] FP32, want[k]: the spawned labels.
 * keep[j] = 1 when the new point stays.  Returns the number rejected.
 */
int orc_territory(int m_s, int d, const float *surv, const int *surv_label, int k, const float *xn,
                  const int *want, int *keep)
{
    int n_rej = 0;
    for (int j = 0; j < k; ++j) {
        float best = INFINITY;
        int bi = -1;
        for (int i = 0; i < m_s; ++i) {
            float s = 0.0f;
            for (int t = 0; t < d; ++t) {
                float diff = xn[(size_t)j * d + t] - surv[(size_t)i * d + t];
                s = fmaf(diff, diff, s);
            }
            if (s < best) { best = s; bi = i; }
        }
        keep[j] = (bi < 0) || (surv_label[bi] == want[j]);
        n_rej += !keep[j];
    }
    return n_rej;
}

/* ------------------------------------------------------------------------- */
/* The GGNS driver (Algorithm 3)                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    double logz, logz_err, logz_skilling_err, info_h;
    long n_iter, n_dead, n_like, n_steps_total, n_fallback, n_region_rejected;
    double dt;
    int n_clusters_final, max_clusters, terminated, status;
} orc_result_t;

typedef struct {
    double lstar, dt, out_frac, logz, log_xl, n_clusters;
} orc_iter_trace_t;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_CAPACITY = 8, ORC_ERR_NOT_DONE = 7 };

/*
 * Full GGNS run.  Dead points (including the final sweep) go to dead_x[cap][d],
 * dead_logl, dead_logw (log prior mass assigned), dead_label; `it_trace` (may be
 * NULL) receives one record per iteration, up to cfg->max_iters.
 */
int orc_run(const orc_cfg_t *cfg, const double *lo, const double *hi, const orc_lik_t *lk,
            orc_result_t *res, long dead_cap, double *dead_x, double *dead_logl,
            double *dead_logw, int *dead_label, orc_iter_trace_t *it_trace)
{
    const int d = lk->d, n_live = cfg->n_live;
    if (n_live < 2 || d < 1) return ORC_ERR_ARG;
    double logdetP = 0.0;
    if (lk->kind == ORC_LIK_DENSE || lk->kind == ORC_LIK_DENSE_MIX) logdetP = orc_logdet_spd(d, lk->precision);
    memset(res, 0, sizeof(*res));
    double *x = (double *)malloc(sizeof(double) * (size_t)n_live * d);
    double *logl = (double *)malloc(sizeof(double) * n_live);
    int *label = (int *)malloc(sizeof(int) * n_live);
    int *order = (int *)malloc(sizeof(int) * n_live);
    int *is_dead = (int *)malloc(sizeof(int) * n_live);
    int *start_slot = (int *)malloc(sizeof(int) * n_live);
    int *new_label = (int *)malloc(sizeof(int) * n_live);
    double *xnew = (double *)malloc(sizeof(double) * (size_t)n_live * d);
    double *lnew = (double *)malloc(sizeof(double) * n_live);
    float *xf = (float *)malloc(sizeof(float) * (size_t)n_live * d);
    int *members = (int *)malloc(sizeof(int) * n_live);
    int *comp = (int *)malloc(sizeof(int) * n_live);
    double *xf_start = (double *)malloc(sizeof(double) * (size_t)n_live * d);
    double *lf_start = (double *)malloc(sizeof(double) * n_live);
    long n_dead = 0, n_like = 0, n_steps_total = 0, n_fallback = 0, n_rejected = 0;
    int status = ORC_OK;

    /* Initialise n_live points from the prior and evaluate their likelihoods. */
    for (int i = 0; i < n_live; ++i) {
        for (int b = 0; 4 * b < d; ++b) {
            uint32_t w[4];
            orc_rng_block(cfg->seed, cfg->run_id, 0, ORC_P_INIT, (uint32_t)i, 0, (uint32_t)b, w);
            for (int t = 0; t < 4 && 4 * b + t < d; ++t) {
                int j = 4 * b + t;
                x[(size_t)i * d + j] = lo[j] + (hi[j] - lo[j]) * orc_u01(w[t]);
            }
        }
        logl[i] = orc_loglik_impl(lk, logdetP, x + (size_t)i * d, NULL);
        label[i] = 0;
        ++n_like;
    }
    orc_stats_t st;
    stats_alloc(&st, n_live);
    st.n[0] = n_live;
    double dt = cfg->dt_init;
    double log_xl_max = ORC_NEG_INF;
    int max_clusters = 1;
    int it;
    int terminated = 0;
    for (it = 0; it < cfg->max_iters; ++it) {
        /* --- cluster finding on every existing cluster (Algorithm 3 + 4) --- */
        if (cfg->clustering) {
            int cap = st.cap;
            int *exists = (int *)malloc(sizeof(int) * cap);
            for (int c = 0; c < cap; ++c) exists[c] = st.alive[c];
            for (int c = 0; c < cap; ++c) {
                if (!exists[c]) continue;
                int m = 0;
                for (int i = 0; i < n_live; ++i) if (label[i] == c) members[m++] = i;
                if (m < 3) continue;
                for (int a = 0; a < m; ++a)
                    for (int t = 0; t < d; ++t) xf[(size_t)a * d + t] = (float)x[(size_t)members[a] * d + t];
                int ncomp = orc_knn_components(m, d, xf, comp);
                if (ncomp <= 1) continue;
                /* parts ordered by their smallest member; part 0 keeps id c */
                int *sz = (int *)calloc(ncomp, sizeof(int));
                int *ids = (int *)malloc(sizeof(int) * ncomp);
                int *root_of = (int *)malloc(sizeof(int) * ncomp);
                int np = 0;
                for (int a = 0; a < m; ++a) if (comp[a] == a) root_of[np++] = a;
                for (int a = 0; a < m; ++a) {
                    int pi = 0;
                    while (root_of[pi] != comp[a]) ++pi;
                    sz[pi]++;
                }
                ids[0] = c;
                int nxt = 0;
                for (int pi = 1; pi < np; ++pi) {
                    while (st.alive[nxt] || nxt == c) ++nxt;
                    ids[pi] = nxt++;
                }
                stats_split(&st, c, np, sz, ids);
                for (int a = 0; a < m; ++a) {
                    int pi = 0;
                    while (root_of[pi] != comp[a]) ++pi;
                    label[members[a]] = ids[pi];
                }
                free(sz); free(ids); free(root_of);
            }
            free(exists);
            int nc = 0;
            for (int c = 0; c < st.cap; ++c) nc += st.alive[c];
            if (nc > max_clusters) max_clusters = nc;
        }
        /* --- kill the n_live // 2 lowest (Algorithm 3), update0-update9 --- */
        const int k = n_live / 2;
        orc_sort_by_logl(n_live, logl, order);
        for (int i = 0; i < n_live; ++i) is_dead[i] = 0;
        double lstar = logl[order[k - 1]];
        for (int j = 0; j < k; ++j) {
            int s = order[j];
            if (n_dead >= dead_cap) { status = ORC_ERR_CAPACITY; break; }
            double lw = stats_kill(&st, label[s], logl[s]);
            if (dead_x) memcpy(dead_x + (size_t)n_dead * d, x + (size_t)s * d, sizeof(double) * d);
            if (dead_logl) dead_logl[n_dead] = logl[s];
            if (dead_logw) dead_logw[n_dead] = lw;
            if (dead_label) dead_label[n_dead] = label[s];
            ++n_dead;
            is_dead[s] = 1;
        }
        if (status != ORC_OK) break;
        /* --- spawn: cluster chosen with probability Xbar_p / sum Xbar, then a
         *     uniform surviving member of that cluster as start point --- */
        double lx_max = ORC_NEG_INF;
        for (int c = 0; c < st.cap; ++c) if (st.alive[c] && st.logXp[c] > lx_max) lx_max = st.logXp[c];
        double total = 0.0;
        for (int c = 0; c < st.cap; ++c) if (st.alive[c]) total += exp(st.logXp[c] - lx_max);
        for (int j = 0; j < k; ++j) {
            uint32_t w[4];
            orc_rng_block(cfg->seed, cfg->run_id, (uint32_t)it, ORC_P_CLUSTER, (uint32_t)j, 0, 0, w);
            double target = orc_u01_53(w[0], w[1]) * total;
            double cum = 0.0;
            int chosen = -1, last_alive = -1;
            for (int c = 0; c < st.cap; ++c) {
                if (!st.alive[c]) continue;
                last_alive = c;
                cum += exp(st.logXp[c] - lx_max);
                if (target < cum) { chosen = c; break; }
            }
            if (chosen < 0) chosen = last_alive;
            int m = 0;
            for (int i = 0; i < n_live; ++i) if (!is_dead[i] && label[i] == chosen) members[m++] = i;
            orc_rng_block(cfg->seed, cfg->run_id, (uint32_t)it, ORC_P_START, (uint32_t)j, 0, 0, w);
            int pick = (int)(((uint64_t)w[0] * (uint64_t)m) >> 32);
            start_slot[j] = members[pick];
            new_label[j] = chosen;
        }
        /* --- HSS for every new point (Algorithm 5) --- */
        long sum_in = 0, sum_out = 0, sum_fold = 0;
        {
            double *xs0 = xf_start;
            double *ls0 = lf_start;
            for (int j = 0; j < k; ++j) {
                memcpy(xs0 + (size_t)j * d, x + (size_t)start_slot[j] * d, sizeof(double) * d);
                ls0[j] = logl[start_slot[j]];
            }
            orc_batch_stats_t bs;
            orc_hss_batch(lk, logdetP, lo, hi, cfg, (uint32_t)it, k, xs0, ls0, lstar, dt, xnew, lnew, NULL, &bs, NULL);
            sum_in = bs.n_in; sum_out = bs.n_out; sum_fold = bs.n_fold;
            n_like += (long)k * bs.t_stop; n_steps_total += (long)k * bs.t_stop;
            n_fallback += bs.n_fallback;
        }
        /* --- a new point in another cluster's region returns its start point --- */
        if (cfg->clustering && cfg->territory) {
            int nc = 0;
            for (int c = 0; c < st.cap; ++c) nc += st.alive[c];
            if (nc > 1) {
                int ms = 0;
                for (int i = 0; i < n_live; ++i) {
                    if (is_dead[i]) continue;
                    for (int t = 0; t < d; ++t) xf[(size_t)ms * d + t] = (float)x[(size_t)i * d + t];
                    members[ms++] = label[i];
                }
                float *xnf = (float *)malloc(sizeof(float) * (size_t)k * d);
                int *keep = (int *)malloc(sizeof(int) * k);
                for (size_t q = 0; q < (size_t)k * d; ++q) xnf[q] = (float)xnew[q];
                n_rejected += orc_territory(ms, d, xf, members, k, xnf, new_label, keep);
                for (int j = 0; j < k; ++j)
                    if (!keep[j]) {
                        memcpy(xnew + (size_t)j * d, x + (size_t)start_slot[j] * d, sizeof(double) * d);
                        lnew[j] = logl[start_slot[j]];
                    }
                free(xnf); free(keep);
            }
        }
        /* --- step-size adaptation from out_frac --- */
        /* (with box_fold and fold_counts, the box's exact reflections count as reflections) */
        const long n_refl = sum_out + ((cfg->box_fold && cfg->fold_counts) ? sum_fold : 0);
        double out_frac = (sum_in + sum_out) > 0 ? (double)n_refl / (double)(sum_in + sum_out) : 0.0;
        if (out_frac > cfg->out_hi) dt *= 0.9;
        else if (out_frac < cfg->out_lo) dt *= 1.1;
        /* --- insert the new points: walker j fills the j-th killed slot --- */
        for (int j = 0; j < k; ++j) {
            int s = order[j];
            memcpy(x + (size_t)s * d, xnew + (size_t)j * d, sizeof(double) * d);
            logl[s] = lnew[j];
            label[s] = new_label[j];
            st.n[new_label[j]] += 1;
        }
        /* --- termination (Section 3, Appendix I; Algorithm 1) --- */
        double lmax = ORC_NEG_INF;
        for (int i = 0; i < n_live; ++i) if (logl[i] > lmax) lmax = logl[i];
        double logX = ORC_NEG_INF;
        for (int c = 0; c < st.cap; ++c) if (st.alive[c]) logX = lae(logX, st.logXp[c]);
        /* the XL-peak statistic on the dead-point sequence: X L* with X the
         * remaining prior volume and L* the last (highest) killed likelihood
         * (the Appendix C definition, L_i X_i / max L_i X_i) */
        double log_xl = logX + lstar;
        if (log_xl > log_xl_max) log_xl_max = log_xl;
        if (it_trace) {
            int nc = 0;
            for (int c = 0; c < st.cap; ++c) nc += st.alive[c];
            it_trace[it].lstar = lstar; it_trace[it].dt = dt; it_trace[it].out_frac = out_frac;
            it_trace[it].logz = st.logZ; it_trace[it].log_xl = log_xl; it_trace[it].n_clusters = nc;
        }
        int stop;
        if (cfg->termination == 0) stop = (log_xl - log_xl_max) < log(cfg->tol);
        else stop = (logX + lmax) < log(cfg->tol) + st.logZ; /* remaining evidence X L_max < tol Z */
        if (stop) { terminated = 1; ++it; break; }
    }
    /* --- final sweep: kill the remaining live points in ascending order with
     *     decreasing n_p (Algorithm 3, last loop) --- */
    if (status == ORC_OK) {
        orc_sort_by_logl(n_live, logl, order);
        for (int j = 0; j < n_live; ++j) {
            int s = order[j];
            if (n_dead >= dead_cap) { status = ORC_ERR_CAPACITY; break; }
            double lw = stats_kill(&st, label[s], logl[s]);
            if (dead_x) memcpy(dead_x + (size_t)n_dead * d, x + (size_t)s * d, sizeof(double) * d);
            if (dead_logl) dead_logl[n_dead] = logl[s];
            if (dead_logw) dead_logw[n_dead] = lw;
            if (dead_label) dead_label[n_dead] = label[s];
            ++n_dead;
        }
    }
    res->logz = st.logZ;
    double var = st.logZ2 - 2.0 * st.logZ;
    res->logz_err = var > 0.0 ? sqrt(var) : 0.0;
    /* Skilling's estimate sqrt(H / n_live), H = sum_i p_i log(L_i / Z) */
    if (dead_logl && dead_logw && status == ORC_OK) {
        double h = 0.0;
        for (long i = 0; i < n_dead; ++i) {
            double lp = dead_logw[i] + dead_logl[i] - st.logZ;
            double p = exp(lp);
            if (p > 0.0) h += p * (dead_logl[i] - st.logZ);
        }
        res->info_h = h;
        res->logz_skilling_err = h > 0.0 ? sqrt(h / n_live) : 0.0;
    }
    res->n_iter = it;
    res->n_dead = n_dead;
    res->n_like = n_like;
    res->n_steps_total = n_steps_total;
    res->n_fallback = n_fallback;
    res->n_region_rejected = n_rejected;
    res->dt = dt;
    res->max_clusters = max_clusters;
    int nc = 0;
    for (int c = 0; c < st.cap; ++c) nc += st.alive[c];
    res->n_clusters_final = nc;
    res->terminated = terminated;
    res->status = (status == ORC_OK && !terminated) ? ORC_ERR_NOT_DONE : status;
    stats_free(&st);
    free(x); free(logl); free(label); free(order); free(is_dead); free(start_slot); free(new_label);
    free(xnew); free(lnew); free(xf); free(members); free(comp); free(xf_start); free(lf_start);
    return res->status;
}

/* Posterior-weighted parameter gradient: d log Z / d mu_k = sum_i p_i d log L(x_i) / d mu_k,
 * p_i = exp(logw_i + logL_i - log Z), the weights held fixed. */
void orc_grad_logz_means(const orc_lik_t *lk, long n, const double *xs, const double *logl,
                         const double *logw, double logz, double *grad)
{
    const int d = lk->d;
    const int K = (lk->kind == ORC_LIK_ISO || lk->kind == ORC_LIK_DENSE) ? 1 : lk->n_comp;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)K * d);
    for (size_t i = 0; i < (size_t)K * d; ++i) grad[i] = 0.0;
    for (long i = 0; i < n; ++i) {
        double p = exp(logw[i] + logl[i] - logz);
        if (!(p > 0.0)) continue;
        orc_loglik_dmeans(lk, xs + (size_t)i * d, tmp);
        for (size_t t = 0; t < (size_t)K * d; ++t) grad[t] += p * tmp[t];
    }
    free(tmp);
}
