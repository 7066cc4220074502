// ggns_api.cu -- host side of libggns: the C ABI of include/ggns.h.
//
// A context holds one or more independent runs.  Device memory is owned by the
// context (cudaMalloc); every iteration of Algorithm 3 is a fixed sequence of
// kernels covering all runs:
//   [k-NN ranks, cluster split]  (Algorithm 4, when clustering is on)
//   selection + Appendix H statistics + spawn   (one CTA per run)
//   HSS phases 0, 1, 2 per walker-tile class     (Algorithm 5)
//   tail: step-size rule and termination          (Algorithm 3)
// ns_run captures several iterations into a CUDA graph and replays it until
// every run has set its done flag, then launches the final sweep.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ggns_iter.cuh"
#include "ggns_tc.cuh"
#include "ggns_kernels.cuh"

using namespace ggns;

namespace {
thread_local std::string g_create_error;
}

namespace ggns {
void set_global_error(const char *msg) { g_create_error = msg ? msg : ""; }
const KindLaunch &kind_launch_iso();
const KindLaunch &kind_launch_mix();
const KindLaunch &kind_launch_dense();
const KindLaunch &kind_launch_densemix();
const KindLaunch &kind_launch_rosen();
const KindLaunch &kind_launch_torus();
const KindLaunch &kind_launch(int kind)
{
    switch (kind) {
    case NS_LIK_ISO_GAUSS: return kind_launch_iso();
    case NS_LIK_MIX_ISO: return kind_launch_mix();
    case NS_LIK_DENSE_GAUSS: return kind_launch_dense();
    case NS_LIK_DENSE_MIX: return kind_launch_densemix();
    case NS_LIK_TORUS: return kind_launch_torus();
    default: return kind_launch_rosen();
    }
}
}  // namespace ggns

namespace {

constexpr int GRAPH_ITERS = 16;
constexpr size_t SMEM_LIMIT = 200 * 1024;
constexpr size_t COOP_SMEM_LIMIT = 227 * 1024;  // one CTA per SM: the whole opt-in shared memory
constexpr int NOISE_BLOCKS_PER_RUN = 64;

struct RunClass {
    int kind, tile;
    int *runs_dev = nullptr;
    std::vector<int> runs;
    int max_k = 0, max_n = 0;
    size_t smem = 0;
    int prec_in_smem = 0;
    int single = 0;    // HSS in one pass (every walker block resident at once)
    int fallback = 1;  // three-phase kernels after the single pass (records shorter than n_steps)
    int coop = 0;      // dense kinds with P outside shared memory, the CTA-cooperative single pass:
                       // 1 contraction on CUDA cores, 2 on the tensor cores
    int coop_tr = 0;   // rows of P per shared-memory tile
    size_t coop_smem = 0;
};

// Runs advanced together by one CUDA graph on one stream.  Different groups run
// on different streams (GGNS_RUNS_PER_GROUP runs each); the default is a single
// group, because concurrent groups share the SMs and the walkers of one group's
// single-pass HSS then stop being co-resident.
struct Group {
    int r0 = 0, nr = 0, max_n = 0, max_k = 0, max_d = 0;
    std::vector<RunClass> classes;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev[GRAPH_ITERS][2] = {};
    cudaEvent_t done_ev = nullptr;
    // the statistics update runs on a second stream, beside the HSS phases
    cudaStream_t ev_stream = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // the momentum noise of the single-pass HSS is drawn on a third stream
    cudaStream_t nz_stream = nullptr;
    cudaEvent_t nz_fork_ev = nullptr, nz_join_ev = nullptr;
    // the iteration's tail runs on the noise stream after the pick, beside the next k-NN
    cudaEvent_t pick_ev = nullptr, tail_ev = nullptr;
    int launches_per_iter = 0;    // kernels of the last launched iteration
    int launches_per_replay = 0;  // kernels of one replay of the captured graph
};

struct DeadHost {
    float *x = nullptr, *logl = nullptr;
    double *logw = nullptr;
    int *label = nullptr;
    long cap = 0;
};

}  // namespace

struct ns_ctx {
    int n_runs = 0;
    std::vector<RunDesc> desc;
    std::vector<DeadHost> dead;
    std::vector<std::vector<double>> prec64;  // FP64 precision of dense mixtures (P mu_k on new means)
    DevCtx dc{};
    RunDesc *desc_dev = nullptr;
    RunState *state_dev = nullptr;
    Stats *stats_dev = nullptr;
    float *fa = nullptr;
    float *logl = nullptr;
    int *label = nullptr, *order = nullptr, *start_slot = nullptr, *new_label = nullptr, *wint = nullptr, *nbr = nullptr;
    float *wres = nullptr;
    unsigned long long *lastkey = nullptr;
    long fa_len = 0, pt_len = 0, w_len = 0;
    std::vector<RunClass> classes;
    std::vector<Group> groups;
    cudaEvent_t start_ev = nullptr;
    double hss_ms_sum = 0.0;
    bool any_clustering = false;
    bool any_territory = false;  // some run keeps new points in their cluster's region
    bool any_midpoint = false;   // some run takes the time-reversible step (its picks are evaluated)
    int max_n = 0, max_d = 0;
    size_t sel_smem = 0, knn_smem = 0, cl_smem = 0, sort_smem = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    std::string err;
    int device = 0;
    std::vector<ns_config> cfg;
    // profiling: CUDA events around the HSS phases of every captured iteration
    cudaEvent_t ev[GRAPH_ITERS][2] = {};
    double hss_ms = 0.0;
    long hss_iters = 0, launches = 0, replays = 0;
    // single-pass HSS records (one row per walker-step, rec_len rows per walker)
    RecView rec{};
    long *rec_base_dev = nullptr;
    int hss_mode = 0;  // 0 automatic, 1 single pass where resident, 3 always three phases
    int launches_per_iter = 0;
    // scratch for the posterior kernels (grown on demand, reused)
    double *scratch = nullptr;
    size_t scratch_len = 0;
};

namespace {

ns_status fail(ns_ctx *c, ns_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return st;
}

#define CU(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? NS_ERR_OOM : NS_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
    } while (0)

// Device scratch of one call, freed when the call returns on every path.
struct DevScratch {
    void *p = nullptr;
    DevScratch() = default;
    DevScratch(const DevScratch &) = delete;
    DevScratch &operator=(const DevScratch &) = delete;
    ~DevScratch()
    {
        if (p) cudaFree(p);
    }
    template <typename T>
    T *as() const
    {
        return static_cast<T *>(p);
    }
};

int default_tile(int kind, int d)
{
    (void)kind;
    if (d <= 2) return 0;
    if (d <= 4) return 1;
    if (d <= 8) return 2;
    if (d <= 16) return 3;
    if (d <= 32) return 4;
    if (d <= 64) return 5;
    if (d <= 128) return 6;
    if (d <= 256) return 7;
    return 8;
}

// The walker tile a configuration asks for (cfg.tile = id + 1), or -1 for the
// library's table; a tile too narrow for d is refused by validate().
int cfg_tile(const ns_config &c) { return (c.tile >= 1 && c.tile <= N_TILES) ? c.tile - 1 : -1; }

// log det of an SPD matrix (unpivoted Cholesky); NAN if not positive definite.
double host_logdet(int d, const double *a)
{
    std::vector<double> l((size_t)d * d, 0.0);
    double ld = 0.0;
    for (int j = 0; j < d; ++j) {
        double s = a[(size_t)j * d + j];
        for (int k = 0; k < j; ++k) s -= l[(size_t)j * d + k] * l[(size_t)j * d + k];
        if (!(s > 0.0)) return NAN;
        const double ljj = std::sqrt(s);
        l[(size_t)j * d + j] = ljj;
        ld += 2.0 * std::log(ljj);
        for (int i = j + 1; i < d; ++i) {
            double t = a[(size_t)i * d + j];
            for (int k = 0; k < j; ++k) t -= l[(size_t)i * d + k] * l[(size_t)j * d + k];
            l[(size_t)i * d + j] = t / ljj;
        }
    }
    return ld;
}

ns_status validate(const ns_prior_box &b, const ns_likelihood_spec &lk, const ns_config &cfg)
{
    if (b.d < 1 || b.d > DMAX || lk.d != b.d || !b.lo || !b.hi)
        return fail(nullptr, NS_ERR_ARG, "dimension must be in [1, %d] and match the prior box", DMAX);
    for (int i = 0; i < b.d; ++i)
        if (!(b.lo[i] < b.hi[i])) return fail(nullptr, NS_ERR_ARG, "prior box needs lo < hi (axis %d)", i);
    if (cfg.n_live < 2 || cfg.n_live > NLIVE_MAX) return fail(nullptr, NS_ERR_ARG, "n_live must be in [2, %d]", NLIVE_MAX);
    if (cfg.min_ref < 0 || cfg.max_ref < cfg.min_ref) return fail(nullptr, NS_ERR_ARG, "need 0 <= min_ref <= max_ref");
    if (cfg.n_steps < 1 || cfg.min_steps < 0) return fail(nullptr, NS_ERR_ARG, "need n_steps >= 1, min_steps >= 0");
    if (!(cfg.dt_init > 0.0) || !(cfg.tol > 0.0)) return fail(nullptr, NS_ERR_ARG, "dt_init and tol must be positive");
    if (cfg.noise_mode == 1 && !(cfg.delta_p >= 0.0 && cfg.delta_p <= 1.0))
        return fail(nullptr, NS_ERR_ARG, "noise_mode 1 needs 0 <= delta_p <= 1");
    if (cfg.max_iters < 1) return fail(nullptr, NS_ERR_ARG, "max_iters must be >= 1");
    if (cfg.tile < 0 || cfg.tile > N_TILES) return fail(nullptr, NS_ERR_ARG, "tile must be 0 or a tile id + 1 in [1, %d]", N_TILES);
    if (cfg.tile > 0) {
        const Tile T = tile_of(cfg.tile - 1);
        if (T.g * T.e < b.d) return fail(nullptr, NS_ERR_ARG, "tile %d covers %d < d = %d components", cfg.tile, T.g * T.e, b.d);
    }
    if (cfg.hss_mode < 0 || cfg.hss_mode > 2 || cfg.rec_len < 0 || cfg.noise_ahead < -1 || cfg.runs_per_group < 0)
        return fail(nullptr, NS_ERR_ARG, "launch choices out of range");
    if (cfg.midpoint != 0 && (cfg.box_fold == 0 || cfg.noise_mode != 1 || lk.kind == NS_LIK_TORUS || cfg.hss_mode == 2))
        return fail(nullptr, NS_ERR_ARG, "midpoint needs box_fold 1, noise_mode 1, a non-periodic kind and the single pass");
    const int K = lk.n_comp;
    switch (lk.kind) {
    case NS_LIK_ISO_GAUSS:
    case NS_LIK_MIX_ISO:
        if (K < 1 || K > KMAX_COMP || !lk.means || !lk.sigma) return fail(nullptr, NS_ERR_ARG, "ISO kinds need means and sigma");
        if (lk.kind == NS_LIK_ISO_GAUSS && K != 1) return fail(nullptr, NS_ERR_ARG, "ISO_GAUSS has one component");
        for (int k = 0; k < K; ++k)
            if (!(lk.sigma[k] > 0.0)) return fail(nullptr, NS_ERR_ARG, "sigma must be positive");
        break;
    case NS_LIK_DENSE_GAUSS:
    case NS_LIK_DENSE_MIX:
        if (K < 1 || K > KMAX_COMP || !lk.means || !lk.precision) return fail(nullptr, NS_ERR_ARG, "DENSE kinds need means and precision");
        if (lk.kind == NS_LIK_DENSE_GAUSS && K != 1) return fail(nullptr, NS_ERR_ARG, "DENSE_GAUSS has one component");
        break;
    case NS_LIK_ROSENBROCK:
        if (lk.d < 2) return fail(nullptr, NS_ERR_ARG, "ROSENBROCK needs d >= 2");
        break;
    case NS_LIK_TORUS:
        if (!(lk.torus_c > 0.0) || !std::isfinite(lk.torus_c) || !std::isfinite(lk.torus_alpha) ||
            !std::isfinite(lk.torus_beta))
            return fail(nullptr, NS_ERR_ARG, "TORUS needs finite frequencies and torus_c > 0");
        break;
    default:
        return fail(nullptr, NS_ERR_ARG, "unknown likelihood kind %d", (int)lk.kind);
    }
    return NS_OK;
}

// Parameter block of one run (FP32 copy of the FP64 inputs, see ParLayout).
ns_status build_params(const ns_prior_box &b, const ns_likelihood_spec &lk, int d_pad, std::vector<float> &out,
                       float &lik_const, float &tc_sv, float &tc_inv)
{
    const int d = b.d, K = kind_has_means(lk.kind) ? lk.n_comp : 1;
    const ParLayout L = par_layout(d, d_pad, K, lk.kind);
    out.assign(L.total, 0.f);
    for (int i = 0; i < d; ++i) {
        out[L.lo + i] = (float)b.lo[i];
        out[L.hi + i] = (float)b.hi[i];
    }
    const double log2pi = 1.8378770664093454836;
    lik_const = 0.f;
    tc_sv = tc_inv = 1.f;
    if (!kind_has_means(lk.kind)) return NS_OK;
    for (int k = K; k < comp_slots(K, lk.kind); ++k) out[L.comp_b + k] = -INFINITY;  // padding: weight 0
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < d; ++i) out[L.means + (long)k * d_pad + i] = (float)lk.means[(size_t)k * d + i];
    for (int k = 0; k < K; ++k) {
        const double lw = lk.log_weights ? lk.log_weights[k] : -std::log((double)K);
        if (lk.kind == NS_LIK_ISO_GAUSS || lk.kind == NS_LIK_MIX_ISO) {
            const double s2 = lk.sigma[k] * lk.sigma[k];
            out[L.comp_a + k] = (float)(1.0 / s2);
            out[L.comp_b + k] = (float)((lk.kind == NS_LIK_MIX_ISO ? lw : 0.0) - 0.5 * d * (log2pi + std::log(s2)));
        } else {
            out[L.comp_a + k] = 0.f;
            out[L.comp_b + k] = (float)(lk.kind == NS_LIK_DENSE_MIX ? lw : 0.0);
        }
    }
    if (lk.kind == NS_LIK_DENSE_GAUSS || lk.kind == NS_LIK_DENSE_MIX) {
        const double ld = host_logdet(d, lk.precision);
        if (!std::isfinite(ld)) return fail(nullptr, NS_ERR_ARG, "precision matrix is not positive definite");
        lik_const = (float)(0.5 * ld - 0.5 * d * log2pi);
        for (int j = 0; j < d; ++j)
            for (int i = 0; i < d; ++i) out[L.prec + (long)j * d_pad + i] = (float)lk.precision[(size_t)j * d + i];
        if (lk.kind == NS_LIK_DENSE_MIX) {
            for (int k = 0; k < K; ++k)
                for (int i = 0; i < d; ++i) {
                    double s = 0.0;
                    for (int j = 0; j < d; ++j) s += lk.precision[(size_t)i * d + j] * lk.means[(size_t)k * d + j];
                    out[L.pmu + (long)k * d_pad + i] = (float)s;
                }
        }
        if (tc_layout(lk.kind, d_pad)) {
            // s_p P = P1 + 2^-11 P2 in FP16: s_p = 2^ep puts the largest |P_ij| just below 2^13,
            // P1 is s_p P rounded to nearest, P2 the remainder times 2^11 rounded to nearest.
            // The walkers scale v by s_v = 2^ev, chosen so that |v| up to twice the box's largest
            // coordinate stays below 2^13 (v = x - mu, or x for the mixture).  K-step j of 16
            // columns holds, for each 128-row tile m, the rows in core matrices of 8 rows x 8
            // columns: row r, column kk at half (r/8) 128 + (kk/8) 64 + (r%8) 8 + kk%8.
            double pmax = 0.0, bmax = 0.0;
            for (size_t i = 0; i < (size_t)d * d; ++i) pmax = std::max(pmax, std::fabs(lk.precision[i]));
            for (int i = 0; i < d; ++i) bmax = std::max(bmax, std::max(std::fabs(b.lo[i]), std::fabs(b.hi[i])));
            int e_p = 0, e_v = 0;
            std::frexp(pmax, &e_p);  // pmax < 2^e_p
            std::frexp(bmax > 0.0 ? 2.0 * bmax : 1.0, &e_v);
            const int ep = 13 - e_p, ev = 13 - e_v;
            if (ep + ev < -100 || ep + ev > 100)
                return fail(nullptr, NS_ERR_ARG, "precision or box out of the range of the tensor-core split");
            tc_sv = (float)std::ldexp(1.0, ev);
            tc_inv = (float)std::ldexp(1.0, -(ep + ev));
            __half *h = reinterpret_cast<__half *>(out.data() + L.ptc);
            const int mt = d_pad / 128, ks = d_pad / 16;
            for (int j = 0; j < ks; ++j)
                for (int m = 0; m < mt; ++m)
                    for (int r = 0; r < 128; ++r)
                        for (int kk = 0; kk < 16; ++kk) {
                            const int row = m * 128 + r, col = 16 * j + kk;
                            const double p =
                                (row < d && col < d) ? std::ldexp(lk.precision[(size_t)row * d + col], ep) : 0.0;
                            const __half p1 = __double2half(p);
                            const __half p2 = __double2half(std::ldexp(p - (double)__half2float(p1), 11));
                            const long at = (r / 8) * 128 + ((kk / 8) * 64) + (r % 8) * 8 + (kk % 8);
                            const long blk = (long)j * 2 * mt * 2048;
                            h[blk + (long)m * 2048 + at] = p1;
                            h[blk + (long)mt * 2048 + (long)m * 2048 + at] = p2;
                        }
        }
    }
    return NS_OK;
}

size_t kind_smem(const RunDesc &D, int pis, int G)
{
    size_t f = (size_t)param_smem_floats(D, pis) + (size_t)(HSS_THREADS / G) * D.d_pad + 8;
    const int K = (D.kind == NS_LIK_ISO_GAUSS || D.kind == NS_LIK_DENSE_GAUSS) ? 1 : D.n_comp;
    return f * 4 + (size_t)K * D.d * 8 + 32;
}

ns_status alloc_dead(ns_ctx *ctx, int r, long cap)
{
    RunDesc &D = ctx->desc[r];
    DeadHost nd;
    nd.cap = cap;
    CU(cudaMalloc(&nd.x, sizeof(float) * (size_t)cap * D.d_pad));
    CU(cudaMalloc(&nd.logl, sizeof(float) * (size_t)cap));
    CU(cudaMalloc(&nd.logw, sizeof(double) * (size_t)cap));
    CU(cudaMalloc(&nd.label, sizeof(int) * (size_t)cap));
    DeadHost &od = ctx->dead[r];
    if (od.cap > 0) {
        // keep the rows written so far
        RunState st;
        CU(cudaMemcpyAsync(&st, ctx->state_dev + r, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        const long n = std::min(st.n_dead, od.cap);
        CU(cudaMemcpyAsync(nd.x, od.x, sizeof(float) * (size_t)n * D.d_pad, cudaMemcpyDeviceToDevice, ctx->stream));
        CU(cudaMemcpyAsync(nd.logl, od.logl, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
        CU(cudaMemcpyAsync(nd.logw, od.logw, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
        CU(cudaMemcpyAsync(nd.label, od.label, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    D.dead_x = nd.x;
    D.dead_logl = nd.logl;
    D.dead_logw = nd.logw;
    D.dead_label = nd.label;
    D.dead_cap = cap;
    D.dead_off = 0;
    CU(cudaMemcpyAsync(ctx->desc_dev + r, &D, sizeof(RunDesc), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (od.cap > 0) {
        cudaFree(od.x);
        cudaFree(od.logl);
        cudaFree(od.logw);
        cudaFree(od.label);
    }
    od = nd;
    return NS_OK;
}

// Make room for `iters` more iterations of every unfinished run.
ns_status ensure_dead_capacity(ns_ctx *ctx, int iters, const std::vector<RunState> &st)
{
    for (int r = 0; r < ctx->n_runs; ++r) {
        if (st[r].final_done) continue;
        const RunDesc &D = ctx->desc[r];
        const long need = st[r].n_dead + (long)iters * D.k + D.n_live;
        if (need > D.dead_cap) {
            long cap = std::max(need, 2 * D.dead_cap);
            ns_status s = alloc_dead(ctx, r, cap);
            if (s != NS_OK) return s;
        }
    }
    return NS_OK;
}

// The termination test of the previous iteration, once its statistics are in.
ns_status launch_term_join(ns_ctx *ctx, Group &g, cudaStream_t s)
{
    CU(cudaStreamWaitEvent(s, g.tail_ev, 0));
    CU(cudaStreamWaitEvent(s, g.join_ev, 0));
    CU(launch_term(ctx->dc, g.r0, g.nr, s));
    return NS_OK;
}

// The momentum noise of the next iteration, drawn ahead on the noise stream (the
// cooperative walks draw theirs where they use it).
static ns_status launch_noise_ahead(ns_ctx *ctx, Group &g, int &n)
{
    for (auto &cl : g.classes)
        if (cl.single && !cl.coop) {
            CU(launch_noise(ctx->dc, cl.runs_dev, (int)cl.runs.size(), NOISE_BLOCKS_PER_RUN, ctx->rec,
                            ctx->rec_base_dev, g.nz_stream));
            ++n;
        }
    CU(cudaEventRecord(g.nz_join_ev, g.nz_stream));
    return NS_OK;
}

// One iteration of Algorithm 3 for the runs of group g, from the k-NN to the pick,
// on stream s.  Unless `first`, the previous iteration's tail (on the noise
// stream) and statistics (on the second stream) are joined after this
// iteration's k-NN, and its termination test runs then.  The tail and, unless
// `last`, the next iteration's noise follow the pick on the noise stream, beside
// the next k-NN.  A launch sequence ends with launch_term_join.
ns_status launch_iteration(ns_ctx *ctx, Group &g, cudaStream_t s, int ev_slot, bool first, bool last)
{
    const DevCtx &C = ctx->dc;
    int n = 0;
    bool any_single = false;
    for (auto &cl : g.classes) any_single |= (cl.single != 0 && !cl.coop);
    const bool noise_ahead = any_single && ctx->rec.nT > 0;
    if (noise_ahead && first) {
        // fork: this iteration's momentum noise beside cluster finding and selection
        CU(cudaEventRecord(g.nz_fork_ev, s));
        CU(cudaStreamWaitEvent(g.nz_stream, g.nz_fork_ev, 0));
        ns_status ns = launch_noise_ahead(ctx, g, n);
        if (ns != NS_OK) return ns;
    }
    if (ctx->any_clustering) {
        CU(launch_knn(C, g.r0, g.nr, g.max_n, ctx->knn_smem, s));
        ++n;
    }
    // the previous iteration's tail and termination test once its statistics are in,
    // then cluster finding and selection: one kernel per run
    if (!first) {
        CU(cudaStreamWaitEvent(s, g.tail_ev, 0));
        CU(cudaStreamWaitEvent(s, g.join_ev, 0));
    }
    CU(launch_term_cluster_sort(C, g.r0, g.nr, ctx->lastkey, std::max(ctx->cl_smem, ctx->sort_smem), !first,
                                ctx->any_clustering, s));
    ++n;
    // fork: the FP64 statistics of this iteration's kills beside the HSS phases
    // (the timing events around the HSS are recorded on the side streams at the same
    // points of the chain, so that no event node sits between two of its kernels)
    CU(cudaEventRecord(g.fork_ev, s));
    CU(cudaStreamWaitEvent(g.ev_stream, g.fork_ev, 0));
    if (ev_slot >= 0) CU(cudaEventRecordWithFlags(g.ev[ev_slot][0], g.ev_stream, cudaEventRecordExternal));
    CU(launch_evidence(C, g.r0, g.nr, ctx->sel_smem, g.ev_stream));
    CU(cudaEventRecord(g.join_ev, g.ev_stream));
    ++n;
    if (noise_ahead) CU(cudaStreamWaitEvent(s, g.nz_join_ev, 0));
    // single pass where every walker block of the class is resident, then the
    // three phases (for single-pass classes only if the records overflowed)
    for (auto &cl : g.classes)
        if (cl.single) {
            if (cl.coop)
                CU(kind_launch(cl.kind).hss1_coop(cl.tile, C, cl.runs_dev, (int)cl.runs.size(), cl.max_k, ctx->rec,
                                                  ctx->rec_base_dev, cl.coop_smem, cl.coop_tr, s));
            else
                CU(kind_launch(cl.kind).hss1(cl.tile, C, cl.runs_dev, (int)cl.runs.size(), cl.max_k, ctx->rec,
                                             ctx->rec_base_dev, cl.smem, cl.prec_in_smem, s));
            ++n;
        }
    for (auto &cl : g.classes)
        if (cl.single) {
            CU(launch_hss_pick(C, cl.runs_dev, (int)cl.runs.size(), cl.max_k, ctx->rec, ctx->rec_base_dev, s));
            ++n;
        }
    // the reversible step: the drawn states are tested against L* (outside: the start point)
    if (ctx->any_midpoint)
        for (auto &cl : g.classes)
            if (cl.single) {
                CU(kind_launch(cl.kind).eval_new(cl.tile, C, cl.runs_dev, (int)cl.runs.size(), cl.max_k, cl.smem,
                                                 cl.prec_in_smem, s));
                ++n;
            }
    for (int phase = 0; phase < 3; ++phase)
        for (auto &cl : g.classes) {
            if (cl.single && !cl.fallback) continue;  // records cover n_steps: no overflow
            CU(kind_launch(cl.kind).hss(cl.tile, C, cl.runs_dev, (int)cl.runs.size(), cl.max_k,
                                        cl.single ? (phase | 4) : phase, cl.smem, cl.prec_in_smem, s));
            ++n;
        }
    // a new point that landed in another cluster's region returns its start point
    if (ctx->any_territory) {
        CU(launch_territory(C, g.r0, g.nr, g.max_k, g.max_d, s));
        ++n;
    }
    // fork: the tail (step size, counters, iteration count), then the next iteration's noise
    CU(cudaEventRecord(g.pick_ev, s));
    CU(cudaStreamWaitEvent(g.nz_stream, g.pick_ev, 0));
    if (ev_slot >= 0) CU(cudaEventRecordWithFlags(g.ev[ev_slot][1], g.nz_stream, cudaEventRecordExternal));
    CU(launch_tail(C, g.r0, g.nr, g.nz_stream));
    CU(cudaEventRecord(g.tail_ev, g.nz_stream));
    ++n;
    if (noise_ahead && !last) {
        ns_status ns = launch_noise_ahead(ctx, g, n);
        if (ns != NS_OK) return ns;
    }
    g.launches_per_iter = n;
    return NS_OK;
}

// Initial state and statistics of every run (eqs. ini0-ini11: one cluster, X = X^2 = 1).
ns_status init_state(ns_ctx *ctx)
{
    const int n_runs = ctx->n_runs;
    std::vector<RunState> st(n_runs);
    std::vector<Stats> sts(n_runs);
    for (int r = 0; r < n_runs; ++r) {
        RunState &S = st[r];
        memset(&S, 0, sizeof S);
        S.dt = ctx->cfg[r].dt_init;
        S.log_xl = S.log_xl_max = -INFINITY;
        S.logz = S.logz2 = -INFINITY;
        S.n_like = ctx->desc[r].n_live;
        S.n_clusters = S.max_clusters = 1;
        Stats &T = sts[r];
        for (int c = 0; c < CMAX; ++c) {
            T.logZp[c] = T.logZp2[c] = T.logZXp[c] = T.logZpXp[c] = T.logXp[c] = T.logXp2[c] = -INFINITY;
            T.n[c] = 0;
            T.alive[c] = 0;
        }
        for (int i = 0; i < CMAX * CMAX; ++i) T.logXX[i] = -INFINITY;
        T.alive[0] = 1;
        T.n[0] = ctx->desc[r].n_live;
        T.logXp[0] = 0.0;
        T.logXp2[0] = 0.0;
    }
    CU(cudaMemcpyAsync(ctx->state_dev, st.data(), sizeof(RunState) * n_runs, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->stats_dev, sts.data(), sizeof(Stats) * n_runs, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return NS_OK;
}

ns_status draw_prior(ns_ctx *ctx)
{
    for (auto &rc : ctx->classes) {
        CU(kind_launch(rc.kind).prior(rc.tile, ctx->dc, rc.runs_dev, (int)rc.runs.size(), rc.max_n, rc.smem,
                                      rc.prec_in_smem, ctx->stream));
        ++ctx->launches;
    }
    return NS_OK;
}

ns_status ensure_scratch(ns_ctx *ctx, size_t n)
{
    if (ctx->scratch_len >= n) return NS_OK;
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_len = 0;
    CU(cudaMalloc(&ctx->scratch, sizeof(double) * n));
    ctx->scratch_len = n;
    return NS_OK;
}

ns_status read_states(ns_ctx *ctx, std::vector<RunState> &st)
{
    st.resize(ctx->n_runs);
    CU(cudaMemcpyAsync(st.data(), ctx->state_dev, sizeof(RunState) * ctx->n_runs, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return NS_OK;
}

ns_status finish_runs(ns_ctx *ctx)
{
    CU(launch_final(ctx->dc, 0, ctx->n_runs, ctx->sel_smem, ctx->stream));
    ++ctx->launches;
    CU(cudaStreamSynchronize(ctx->stream));
    return NS_OK;
}

}  // namespace

// ========================================================================
// C ABI
// ========================================================================
extern "C" {

void ns_config_default(ns_config *c)
{
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->n_live = 200;
    c->n_steps = 1000;
    c->min_steps = 0;
    c->dt_init = 0.1;
    c->delta_p = 0.5;
    c->tol = 0.01;
    c->min_ref = 1;
    c->max_ref = 3;
    c->prune_after = 10;
    c->termination = 0;
    c->clustering = 1;
    c->noise_mode = 1;
    c->out_lo = 0.05;
    c->out_hi = 0.15;
    c->seed = 0;
    c->run_id = 0;
    c->max_iters = 100000;
    c->dead_cap = 0;
    c->noise_inside = 1;
    c->pick_all = 1;
    c->territory = 1;
    c->box_fold = 0;
    c->fold_counts = 0;
}

const char *ns_last_error(const ns_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

ns_status ns_batch_create(int n_runs, const ns_prior_box *box, const ns_likelihood_spec *lik, const ns_config *cfg,
                          ns_ctx **out)
{
    ns_ctx *ctx = nullptr;
    if (!out || n_runs < 1 || !box || !lik || !cfg) return fail(nullptr, NS_ERR_ARG, "invalid arguments to ns_batch_create");
    *out = nullptr;
    for (int r = 0; r < n_runs; ++r) {
        ns_status s = validate(box[r], lik[r], cfg[r]);
        if (s != NS_OK) return s;
    }
    ctx = new ns_ctx();
    ctx->n_runs = n_runs;
    cudaGetDevice(&ctx->device);
    ctx->desc.resize(n_runs);
    ctx->dead.resize(n_runs);
    std::vector<std::vector<float>> pars(n_runs);
    long fa = 0, pt = 0, w = 0;
    for (int r = 0; r < n_runs; ++r) {
        RunDesc &D = ctx->desc[r];
        memset(&D, 0, sizeof D);
        const ns_config &c = cfg[r];
        D.d = box[r].d;
        D.kind = lik[r].kind;
        D.n_comp = kind_has_means(lik[r].kind) ? lik[r].n_comp : 1;
        const int t = cfg_tile(c);
        D.tile = (t >= 0) ? t : default_tile(D.kind, D.d);
        const Tile T = tile_of(D.tile);
        D.d_pad = T.g * T.e;
        D.n_live = c.n_live;
        D.k = c.n_live / 2;
        D.n_steps = c.n_steps;
        D.min_steps = c.min_steps;
        D.min_ref = c.min_ref;
        D.max_ref = c.max_ref;
        D.prune_after = c.prune_after;
        D.termination = c.termination;
        D.clustering = c.clustering;
        D.noise_mode = c.noise_mode;
        D.noise_inside = c.noise_inside ? 1 : 0;
        D.pick_all = c.pick_all ? 1 : 0;
        D.territory = c.territory ? 1 : 0;
        D.keep_last = c.keep_last ? 1 : 0;
        D.box_fold = c.box_fold ? 1 : 0;
        D.fold_counts = c.fold_counts ? 1 : 0;
        D.midpoint = c.midpoint ? 1 : 0;
        D.delta_p = (float)c.delta_p;
        D.keep = (float)std::sqrt(std::max(0.0, 1.0 - c.delta_p * c.delta_p));
        D.rosen_scale = (float)lik[r].rosen_scale;
        D.torus_a = (float)lik[r].torus_alpha;
        D.torus_b = (float)lik[r].torus_beta;
        D.torus_c = (float)lik[r].torus_c;
        D.log_tol = std::log(c.tol);
        D.out_lo = c.out_lo;
        D.out_hi = c.out_hi;
        D.dt_init = c.dt_init;
        const uint32_t rid = c.run_id;
        D.key0 = (uint32_t)c.seed;
        D.key1 = (uint32_t)(c.seed >> 32) ^ rid;
        D.max_iters = c.max_iters;
        ns_status s = build_params(box[r], lik[r], D.d_pad, pars[r], D.lik_const, D.tc_sv, D.tc_inv);
        if (s != NS_OK) {
            delete ctx;
            return s;
        }
        ctx->prec64.emplace_back();
        if (lik[r].kind == NS_LIK_DENSE_MIX)
            ctx->prec64.back().assign(lik[r].precision, lik[r].precision + (size_t)D.d * D.d);
        D.x_off = fa;
        fa += (long)D.n_live * D.d_pad;
        D.ws_off = fa;
        fa += (long)D.k * 3 * D.d_pad;
        D.par_off = fa;
        fa += (long)pars[r].size();
        fa = (fa + 3) & ~3L;
        D.pt_off = pt;
        D.nbr_off = pt * KNN_K;
        pt += D.n_live;
        D.w_off = w;
        w += D.k;
        ctx->any_clustering |= (D.clustering != 0);
        ctx->any_territory |= (D.clustering != 0 && D.territory != 0);
        ctx->any_midpoint |= (D.midpoint != 0);
        ctx->max_n = std::max(ctx->max_n, D.n_live);
        ctx->max_d = std::max(ctx->max_d, D.d);
    }
    ctx->fa_len = fa;
    ctx->pt_len = pt;
    ctx->w_len = w;
    ns_status s;
#define CK(call)                        \
    do {                                \
        s = (call);                     \
        if (s != NS_OK) {               \
            g_create_error = ctx->err;  \
            ns_destroy(ctx);            \
            return s;                   \
        }                               \
    } while (0)
    auto setup = [&]() -> ns_status {
        CU(cudaStreamCreateWithFlags(&ctx->graph_stream, cudaStreamNonBlocking));
        CU(cudaMalloc(&ctx->desc_dev, sizeof(RunDesc) * n_runs));
        CU(cudaMalloc(&ctx->state_dev, sizeof(RunState) * n_runs));
        CU(cudaMalloc(&ctx->stats_dev, sizeof(Stats) * n_runs));
        CU(cudaMalloc(&ctx->fa, sizeof(float) * fa));
        CU(cudaMemset(ctx->fa, 0, sizeof(float) * fa));
        CU(cudaMalloc(&ctx->logl, sizeof(float) * pt));
        CU(cudaMalloc(&ctx->label, sizeof(int) * pt));
        CU(cudaMalloc(&ctx->order, sizeof(int) * pt));
        CU(cudaMalloc(&ctx->nbr, sizeof(int) * pt * KNN_K));
        CU(cudaMalloc(&ctx->lastkey, sizeof(unsigned long long) * pt));
        CU(cudaMalloc(&ctx->start_slot, sizeof(int) * w));
        CU(cudaMalloc(&ctx->new_label, sizeof(int) * w));
        CU(cudaMalloc(&ctx->wint, sizeof(int) * w * WINT));
        CU(cudaMemset(ctx->wint, 0, sizeof(int) * w * WINT));
        CU(cudaMalloc(&ctx->wres, sizeof(float) * w));
        for (int r = 0; r < n_runs; ++r)
            CU(cudaMemcpy(ctx->fa + ctx->desc[r].par_off, pars[r].data(), sizeof(float) * pars[r].size(),
                          cudaMemcpyHostToDevice));
        CU(cudaMemcpy(ctx->desc_dev, ctx->desc.data(), sizeof(RunDesc) * n_runs, cudaMemcpyHostToDevice));
        return NS_OK;
    };
    ctx->cfg.assign(cfg, cfg + n_runs);
    CK(setup());
    CK(init_state(ctx));
    DevCtx &C = ctx->dc;
    C.n_runs = n_runs;
    C.desc = ctx->desc_dev;
    C.state = ctx->state_dev;
    C.stats = ctx->stats_dev;
    C.fa = ctx->fa;
    C.logl = ctx->logl;
    C.label = ctx->label;
    C.order = ctx->order;
    C.start_slot = ctx->start_slot;
    C.new_label = ctx->new_label;
    C.wint = ctx->wint;
    C.wres_logl = ctx->wres;
    C.nbr = ctx->nbr;
    // dead arenas: one allocation per run, grown between graph replays
    for (int r = 0; r < n_runs; ++r) {
        const RunDesc &D = ctx->desc[r];
        long cap = cfg[r].dead_cap > 0 ? cfg[r].dead_cap : (long)D.n_live * 64 + D.k * GRAPH_ITERS;
        CK(alloc_dead(ctx, r, cap));
    }
    // walker-tile classes
    std::map<std::pair<int, int>, int> cls;
    for (int r = 0; r < n_runs; ++r) {
        const RunDesc &D = ctx->desc[r];
        auto key = std::make_pair(D.kind, D.tile);
        if (!cls.count(key)) {
            cls[key] = (int)ctx->classes.size();
            RunClass rc;
            rc.kind = D.kind;
            rc.tile = D.tile;
            ctx->classes.push_back(rc);
        }
        RunClass &rc = ctx->classes[cls[key]];
        rc.runs.push_back(r);
        rc.max_k = std::max(rc.max_k, D.k);
        rc.max_n = std::max(rc.max_n, D.n_live);
    }
    for (auto &rc : ctx->classes) {
        const Tile T = tile_of(rc.tile);
        size_t need_in = 0, need_out = 0;
        for (int r : rc.runs) {
            need_in = std::max(need_in, kind_smem(ctx->desc[r], 1, T.g));
            need_out = std::max(need_out, kind_smem(ctx->desc[r], 0, T.g));
        }
        rc.prec_in_smem = need_in <= SMEM_LIMIT ? 1 : 0;
        rc.smem = rc.prec_in_smem ? need_in : need_out;
        if (rc.smem > SMEM_LIMIT) {
            g_create_error = "likelihood parameters exceed the shared-memory budget";
            ns_destroy(ctx);
            return NS_ERR_ARG;
        }
        auto setup_cls = [&]() -> ns_status {
            CU(cudaMalloc(&rc.runs_dev, sizeof(int) * rc.runs.size()));
            CU(cudaMemcpy(rc.runs_dev, rc.runs.data(), sizeof(int) * rc.runs.size(), cudaMemcpyHostToDevice));
            CU(kind_launch(rc.kind).set_smem(rc.tile, rc.smem));
            return NS_OK;
        };
        CK(setup_cls());
    }
    // single-pass HSS records: GGNS_HSS = 3 keeps the three-phase form, GGNS_REC_LEN
    // sets the records per walker (default n_steps, halved until they fit 8 GiB)
    int n_sm = 0;
    auto smq = [&]() -> ns_status {
        CU(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
        return NS_OK;
    };
    CK(smq());
    {
        ctx->hss_mode = (cfg[0].hss_mode == 2) ? 3 : cfg[0].hss_mode;  // ns_config: 2 = three phases always
        long rec_len = 1l << 30;
        if (cfg[0].rec_len > 0) rec_len = cfg[0].rec_len;
        int max_steps = 0, xs = 0;
        long walkers = 0;
        for (int r = 0; r < n_runs; ++r) {
            max_steps = std::max(max_steps, cfg[r].n_steps);
            xs = std::max(xs, ctx->desc[r].d_pad);
            walkers += ctx->desc[r].k;
        }
        rec_len = std::min<long>(rec_len, max_steps);
        const long budget = 8l << 30;
        const long row_bytes = (long)xs * 4 + 12;
        while (rec_len > 16 && walkers * rec_len * row_bytes > budget) rec_len /= 2;
        if (ctx->hss_mode != 3 && walkers * rec_len * row_bytes <= budget) {
            auto mkrec = [&]() -> ns_status {
                const long rows = walkers * rec_len;
                CU(cudaMalloc(&ctx->rec.meta, sizeof(uint2) * rows));
                CU(cudaMalloc(&ctx->rec.ll, sizeof(float) * rows));
                CU(cudaMalloc(&ctx->rec.x, sizeof(float) * rows * xs));
                std::vector<long> base(n_runs);
                long acc = 0;
                for (int r = 0; r < n_runs; ++r) {
                    base[r] = acc;
                    acc += (long)ctx->desc[r].k * rec_len;
                }
                CU(cudaMalloc(&ctx->rec_base_dev, sizeof(long) * n_runs));
                CU(cudaMemcpy(ctx->rec_base_dev, base.data(), sizeof(long) * n_runs, cudaMemcpyHostToDevice));
                ctx->rec.rec_len = (int)rec_len;
                ctx->rec.xs = xs;
                // noise drawn ahead: noise_ahead steps per walker (0: the default 128; -1: off)
                long nT = 128;
                if (cfg[0].noise_ahead > 0) nT = cfg[0].noise_ahead;
                else if (cfg[0].noise_ahead < 0) nT = 0;
                nT = std::min<long>(nT, rec_len);
                if (xs % 4 != 0 || walkers * nT * ((long)xs * 4 + 4) > budget) nT = 0;
                if (nT > 0) {
                    CU(cudaMalloc(&ctx->rec.nz, sizeof(float) * walkers * nT * xs));
                    CU(cudaMalloc(&ctx->rec.nsp, sizeof(uint32_t) * walkers * nT));
                }
                ctx->rec.nT = (int)nT;
                return NS_OK;
            };
            CK(mkrec());
        }
    }
    // run groups: one stream and one graph each (runs_per_group runs; default: all runs in one group)
    {
        int per = n_runs;
        if (cfg[0].runs_per_group > 0) per = cfg[0].runs_per_group;
        per = std::max(per, (n_runs + 127) / 128);
        auto mkgroups = [&]() -> ns_status {
            CU(cudaEventCreateWithFlags(&ctx->start_ev, cudaEventDefault));
            for (int r0 = 0; r0 < n_runs; r0 += per) {
                Group g;
                g.r0 = r0;
                g.nr = std::min(per, n_runs - r0);
                std::map<std::pair<int, int>, int> gcls;
                for (int r = g.r0; r < g.r0 + g.nr; ++r) {
                    const RunDesc &D = ctx->desc[r];
                    g.max_n = std::max(g.max_n, D.n_live);
                    g.max_k = std::max(g.max_k, D.k);
                    g.max_d = std::max(g.max_d, D.d);
                    auto key = std::make_pair(D.kind, D.tile);
                    if (!gcls.count(key)) {
                        gcls[key] = (int)g.classes.size();
                        RunClass rc = ctx->classes[cls[key]];
                        rc.runs.clear();
                        rc.runs_dev = nullptr;
                        rc.max_k = rc.max_n = 0;
                        g.classes.push_back(rc);
                    }
                    RunClass &rc = g.classes[gcls[key]];
                    rc.runs.push_back(r);
                    rc.max_k = std::max(rc.max_k, D.k);
                    rc.max_n = std::max(rc.max_n, D.n_live);
                }
                for (auto &rc : g.classes) {
                    CU(cudaMalloc(&rc.runs_dev, sizeof(int) * rc.runs.size()));
                    CU(cudaMemcpy(rc.runs_dev, rc.runs.data(), sizeof(int) * rc.runs.size(), cudaMemcpyHostToDevice));
                    rc.single = 0;
                    if (ctx->rec.rec_len > 0) {
                        int per_sm = 0;
                        CU(kind_launch(rc.kind).hss1_occ(rc.tile, rc.smem, &per_sm));
                        const long gpc = HSS_THREADS / tile_of(rc.tile).g;
                        const long blocks = (rc.max_k + gpc - 1) / gpc * (long)rc.runs.size();
                        rc.single = blocks <= (long)per_sm * n_sm ? 1 : 0;
                        rc.fallback = 0;
                        for (int r : rc.runs) rc.fallback |= (ctx->rec.rec_len < cfg[r].n_steps);
                        // dense likelihoods whose P stays in global memory: the walkers of a CTA share
                        // each tile of P, with the contraction on the tensor cores (coop 0) or on CUDA
                        // cores (coop 1); coop = -1 keeps one read of P per walker-step
                        const bool want = cfg[0].coop >= 0;
                        const bool dense = rc.kind == NS_LIK_DENSE_GAUSS || rc.kind == NS_LIK_DENSE_MIX;
                        // (the tensor-core form also where P would fit in shared memory: d_pad = 128)
                        if (want && dense && (!rc.prec_in_smem || cfg[0].coop == 0) && !rc.fallback &&
                            (rc.tile == 6 || rc.tile == 7 || rc.tile == 8)) {
                            size_t par = 0;
                            int dpm = 0;
                            bool aligned = true;
                            for (int r : rc.runs) {
                                const RunDesc &Dr = ctx->desc[r];
                                par = std::max(par, (size_t)param_smem_floats(Dr, false));
                                dpm = std::max(dpm, Dr.d_pad);
                                const ParLayout Lr = par_layout(Dr.d, Dr.d_pad, Dr.n_comp, Dr.kind);
                                aligned &= ((Dr.par_off + Lr.prec) % 4) == 0;
                            }
                            const long cb = (rc.max_k + COOP_THREADS / 32 - 1) / (COOP_THREADS / 32) *
                                            (long)rc.runs.size();
                            // the contraction on the tensor cores (coop = 0, the default)
                            if (cfg[0].coop == 0 && aligned && tc_layout(rc.kind, dpm)) {
                                const size_t need = 4 * par + tc::plan(dpm).total + 1024;
                                int cps = 0;
                                if (need <= COOP_SMEM_LIMIT) CU(kind_launch(rc.kind).hss1_coop_occ(rc.tile, need, 0, &cps));
                                if (need <= COOP_SMEM_LIMIT && cps > 0 && cb <= (long)cps * n_sm) {
                                    rc.coop = 2;
                                    rc.coop_tr = 0;
                                    rc.coop_smem = need;
                                    rc.single = 1;
                                }
                            }
                            const size_t base = 4 * (par + (size_t)(COOP_THREADS / 32) * dpm) + 16;
                            for (int tr = 64; tr >= 8 && aligned && rc.coop == 0 && !rc.prec_in_smem; tr /= 2) {
                                const size_t need = base + 2 * 4 * (size_t)tr * dpm;
                                if (need > COOP_SMEM_LIMIT) continue;
                                int cps = 0;
                                CU(kind_launch(rc.kind).hss1_coop_occ(rc.tile, need, tr, &cps));
                                if (cps > 0 && cb <= (long)cps * n_sm) {
                                    rc.coop = 1;
                                    rc.coop_tr = tr;
                                    rc.coop_smem = need;
                                    rc.single = 1;
                                }
                                break;
                            }
                        }
                    }
                }
                // the iteration's chain (k-NN, selection, HSS, pick, tail) runs at the highest
                // priority: CTAs of the side streams (noise drawn ahead, statistics) take the SMs
                // only where the chain leaves room, instead of delaying it
                int prio_low = 0, prio_high = 0;
                CU(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
                CU(cudaStreamCreateWithPriority(&g.stream, cudaStreamNonBlocking, prio_high));
                CU(cudaStreamCreateWithPriority(&g.ev_stream, cudaStreamNonBlocking, prio_low));
                CU(cudaStreamCreateWithPriority(&g.nz_stream, cudaStreamNonBlocking, prio_low));
                CU(cudaEventCreateWithFlags(&g.nz_fork_ev, cudaEventDisableTiming));
                CU(cudaEventCreateWithFlags(&g.nz_join_ev, cudaEventDisableTiming));
                CU(cudaEventCreateWithFlags(&g.pick_ev, cudaEventDisableTiming));
                CU(cudaEventCreateWithFlags(&g.tail_ev, cudaEventDisableTiming));
                CU(cudaEventCreateWithFlags(&g.fork_ev, cudaEventDisableTiming));
                CU(cudaEventCreateWithFlags(&g.join_ev, cudaEventDisableTiming));
                for (int i = 0; i < GRAPH_ITERS; ++i)
                    for (int j = 0; j < 2; ++j) CU(cudaEventCreate(&g.ev[i][j]));
                CU(cudaEventCreateWithFlags(&g.done_ev, cudaEventDisableTiming));
                ctx->groups.push_back(g);
            }
            return NS_OK;
        };
        CK(mkgroups());
    }
    // the reversible step needs the single pass with records for every step (the three-phase
    // kernels take the printed step)
    for (auto &g : ctx->groups)
        for (auto &cl : g.classes)
            for (int r : cl.runs)
                if (ctx->desc[r].midpoint && (!cl.single || cl.fallback)) {
                    ns_destroy(ctx);
                    return fail(nullptr, NS_ERR_ARG, "run %d: midpoint needs the single-pass walk with records for "
                                                     "every step (resident walkers, rec_len >= n_steps)", r);
                }
    ctx->sel_smem = select_smem_bytes(ctx->max_n);
    ctx->knn_smem = knn_smem_bytes(ctx->max_d);
    ctx->cl_smem = cluster_smem_bytes(ctx->max_n);
    ctx->sort_smem = sort_smem_bytes(ctx->max_n);
    auto attrs = [&]() -> ns_status {
        CU(prepare_iteration_kernels(ctx->sel_smem, ctx->knn_smem, ctx->cl_smem, ctx->sort_smem));
        return NS_OK;
    };
    CK(attrs());
    // prior draws and their likelihoods (Algorithm 3, first step)
    auto prior = [&]() -> ns_status {
        ns_status ps = draw_prior(ctx);
        if (ps != NS_OK) return ps;
        CU(cudaStreamSynchronize(ctx->stream));
        return NS_OK;
    };
    CK(prior());
#undef CK
    *out = ctx;
    return NS_OK;
}

ns_status ns_create(const ns_prior_box *box, const ns_likelihood_spec *lik, const ns_config *cfg, ns_ctx **out)
{
    return ns_batch_create(1, box, lik, cfg, out);
}

ns_status ns_set_stream(ns_ctx *ctx, void *stream)
{
    if (!ctx) return NS_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return NS_OK;
}

ns_status ns_step(ns_ctx *ctx, int n_iters, int *done)
{
    if (!ctx || n_iters < 0) return NS_ERR_ARG;
    std::vector<RunState> st;
    ns_status s = read_states(ctx, st);
    if (s != NS_OK) return s;
    s = ensure_dead_capacity(ctx, n_iters, st);
    if (s != NS_OK) return s;
    for (auto &g : ctx->groups) {
        for (int i = 0; i < n_iters; ++i) {
            s = launch_iteration(ctx, g, ctx->stream, -1, i == 0, i == n_iters - 1);
            if (s != NS_OK) return s;
            ctx->launches += g.launches_per_iter;
        }
        if (n_iters > 0) {
            s = launch_term_join(ctx, g, ctx->stream);
            if (s != NS_OK) return s;
            ++ctx->launches;
        }
    }
    s = read_states(ctx, st);
    if (s != NS_OK) return s;
    int all = 1;
    for (auto &x : st) all &= x.done;
    if (done) *done = all;
    return NS_OK;
}

ns_status ns_run(ns_ctx *ctx, long max_iters)
{
    if (!ctx) return NS_ERR_ARG;
    std::vector<RunState> st;
    ns_status s = read_states(ctx, st);
    if (s != NS_OK) return s;
    for (auto &g : ctx->groups) {
        if (g.graph) continue;
        // capture GRAPH_ITERS iterations of this group once; kernels of finished runs return at once
        cudaGraph_t gr;
        CU(cudaStreamBeginCapture(g.stream, cudaStreamCaptureModeThreadLocal));
        g.launches_per_replay = 1;  // the termination test that closes the sequence
        for (int i = 0; i < GRAPH_ITERS; ++i) {
            s = launch_iteration(ctx, g, g.stream, i, i == 0, i == GRAPH_ITERS - 1);
            if (s != NS_OK) {
                cudaStreamEndCapture(g.stream, &gr);
                return s;
            }
            g.launches_per_replay += g.launches_per_iter;
        }
        s = launch_term_join(ctx, g, g.stream);
        if (s != NS_OK) {
            cudaStreamEndCapture(g.stream, &gr);
            return s;
        }
        CU(cudaStreamEndCapture(g.stream, &gr));
        CU(cudaGraphInstantiateWithFlags(&g.graph, gr, cudaGraphInstantiateFlagUseNodePriority));
        cudaGraphDestroy(gr);
    }
    long done_iters = 0;
    std::vector<std::pair<float, float>> spans;
    for (;;) {
        int all = 1;
        for (auto &x : st) all &= x.done;
        if (all || done_iters >= max_iters) break;
        s = ensure_dead_capacity(ctx, GRAPH_ITERS, st);
        if (s != NS_OK) return s;
        std::vector<int> it0(ctx->n_runs);
        for (int r = 0; r < ctx->n_runs; ++r) it0[r] = st[r].iter;
        CU(cudaEventRecord(ctx->start_ev, ctx->stream));
        std::vector<int> launched(ctx->groups.size(), 0);
        for (size_t gi = 0; gi < ctx->groups.size(); ++gi) {
            Group &g = ctx->groups[gi];
            bool busy = false;
            for (int r = g.r0; r < g.r0 + g.nr; ++r) busy |= !st[r].done;
            if (!busy) continue;
            launched[gi] = 1;
            CU(cudaStreamWaitEvent(g.stream, ctx->start_ev, 0));
            CU(cudaGraphLaunch(g.graph, g.stream));
            CU(cudaEventRecord(g.done_ev, g.stream));
            CU(cudaStreamWaitEvent(ctx->stream, g.done_ev, 0));
            ctx->launches += g.launches_per_replay;
        }
        done_iters += GRAPH_ITERS;
        s = read_states(ctx, st);
        if (s != NS_OK) return s;
        // HSS activity: union over groups of the intervals between the events around the three phases
        spans.clear();
        for (size_t gi = 0; gi < ctx->groups.size(); ++gi) {
            if (!launched[gi]) continue;
            Group &g = ctx->groups[gi];
            int active = 0;
            for (int r = g.r0; r < g.r0 + g.nr; ++r) active = std::max(active, st[r].iter - it0[r]);
            for (int i = 0; i < active && i < GRAPH_ITERS; ++i) {
                float a = 0.f, b = 0.f;
                if (cudaEventElapsedTime(&a, ctx->start_ev, g.ev[i][0]) == cudaSuccess &&
                    cudaEventElapsedTime(&b, ctx->start_ev, g.ev[i][1]) == cudaSuccess && b >= a) {
                    spans.push_back({a, b});
                    ctx->hss_ms_sum += b - a;
                }
            }
            ctx->hss_iters += active;
        }
        std::sort(spans.begin(), spans.end());
        float cur_a = -1.f, cur_b = -1.f;
        for (auto &sp : spans) {
            if (sp.first > cur_b) {
                if (cur_b > cur_a) ctx->hss_ms += cur_b - cur_a;
                cur_a = sp.first;
                cur_b = sp.second;
            } else {
                cur_b = std::max(cur_b, sp.second);
            }
        }
        if (cur_b > cur_a) ctx->hss_ms += cur_b - cur_a;
        ++ctx->replays;
    }
    int all = 1;
    for (auto &x : st) all &= x.done;
    if (all) {
        s = finish_runs(ctx);
        if (s != NS_OK) return s;
    }
    return NS_OK;
}

ns_status ns_restart(ns_ctx *ctx, uint64_t seed)
{
    if (!ctx) return NS_ERR_ARG;
    for (int r = 0; r < ctx->n_runs; ++r) {
        RunDesc &D = ctx->desc[r];
        ctx->cfg[r].seed = seed;
        D.key0 = (uint32_t)seed;
        D.key1 = (uint32_t)(seed >> 32) ^ ctx->cfg[r].run_id;
    }
    CU(cudaMemcpyAsync(ctx->desc_dev, ctx->desc.data(), sizeof(RunDesc) * ctx->n_runs, cudaMemcpyHostToDevice,
                       ctx->stream));
    ns_status s = init_state(ctx);
    if (s != NS_OK) return s;
    s = draw_prior(ctx);
    if (s != NS_OK) return s;
    CU(cudaStreamSynchronize(ctx->stream));
    return NS_OK;
}

ns_status ns_profile(const ns_ctx *cctx, double *out, int reset)
{
    ns_ctx *ctx = const_cast<ns_ctx *>(cctx);
    if (!ctx || !out) return NS_ERR_ARG;
    out[0] = ctx->hss_ms;
    out[1] = (double)ctx->hss_iters;
    out[2] = (double)ctx->launches;
    out[3] = (double)ctx->replays;
    out[4] = ctx->hss_ms_sum;
    std::vector<RunState> st;
    ns_status rs = read_states(ctx, st);
    if (rs != NS_OK) return rs;
    long over = 0;
    for (auto &x : st) over += x.n_rec_overflow;
    out[5] = (double)over;
    out[6] = ctx->rec.rec_len;
    out[7] = ctx->rec.nT;
    int ncoop = 0, ntc = 0;
    for (auto &g : ctx->groups)
        for (auto &cl : g.classes) {
            ncoop += cl.coop > 0;
            ntc += cl.coop == 2;
        }
    out[8] = ncoop;
    out[9] = ntc;
    if (reset) {
        ctx->hss_ms = ctx->hss_ms_sum = 0.0;
        ctx->hss_iters = ctx->launches = ctx->replays = 0;
    }
    return NS_OK;
}

ns_status ns_result_run(const ns_ctx *cctx, int run, ns_result_t *out)
{
    ns_ctx *ctx = const_cast<ns_ctx *>(cctx);
    if (!ctx || !out || run < 0 || run >= ctx->n_runs) return NS_ERR_ARG;
    RunState S;
    CU(cudaMemcpyAsync(&S, ctx->state_dev + run, sizeof S, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    memset(out, 0, sizeof *out);
    out->logz = S.logz;
    const double var = S.logz2 - 2.0 * S.logz;
    out->logz_err = var > 0.0 ? std::sqrt(var) : 0.0;
    out->n_iter = S.iter;
    out->n_dead = S.n_dead;
    out->n_like = S.n_like;
    out->n_steps_total = S.n_steps_total;
    out->dt = S.dt;
    out->n_clusters = S.n_clusters;
    out->max_clusters = S.max_clusters;
    out->terminated = S.terminated;
    out->status = S.status;
    if (S.final_done && S.n_dead > 0 && std::isfinite(S.logz)) {
        ns_status es = ensure_scratch(ctx, 2 + 2 * 152);
        if (es != NS_OK) return es;
        double *tmp = ctx->scratch;
        CU(launch_info(ctx->dc, run, S.logz, tmp, ctx->stream));
        ctx->launches += 2;
        double h[2];
        CU(cudaMemcpyAsync(h, tmp, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        out->info_h = h[0];
        out->logz_skilling_err = h[0] > 0.0 ? std::sqrt(h[0] / ctx->desc[run].n_live) : 0.0;
    }
    if (!S.final_done && S.status == NS_OK) return NS_ERR_NOT_DONE;
    return (ns_status)S.status;
}

ns_status ns_result(const ns_ctx *ctx, ns_result_t *out) { return ns_result_run(ctx, 0, out); }

ns_status ns_samples(const ns_ctx *cctx, int run, double *x, double *logp, long cap, long *n_out)
{
    ns_ctx *ctx = const_cast<ns_ctx *>(cctx);
    if (!ctx || run < 0 || run >= ctx->n_runs || !n_out) return NS_ERR_ARG;
    RunState S;
    CU(cudaMemcpyAsync(&S, ctx->state_dev + run, sizeof S, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *n_out = S.n_dead;
    if (!x && !logp && cap == 0) return NS_OK;
    if (cap < S.n_dead) return fail(ctx, NS_ERR_CAPACITY, "ns_samples: cap %ld < %ld dead points", cap, S.n_dead);
    const RunDesc &D = ctx->desc[run];
    const long n = S.n_dead;
    DevScratch xs, ls;
    if (x) CU(cudaMalloc(&xs.p, sizeof(double) * (size_t)n * D.d));
    if (logp) CU(cudaMalloc(&ls.p, sizeof(double) * (size_t)n));
    CU(launch_export(ctx->dc, run, D.d, D.d_pad, S.logz, xs.as<double>(), ls.as<double>(), n, ctx->stream));
    if (x) CU(cudaMemcpyAsync(x, xs.p, sizeof(double) * (size_t)n * D.d, cudaMemcpyDeviceToHost, ctx->stream));
    if (logp) CU(cudaMemcpyAsync(logp, ls.p, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return NS_OK;
}

ns_status ns_grad_logz(const ns_ctx *cctx, int run, double *grad, long cap)
{
    ns_ctx *ctx = const_cast<ns_ctx *>(cctx);
    if (!ctx || run < 0 || run >= ctx->n_runs || !grad) return NS_ERR_ARG;
    const RunDesc &D = ctx->desc[run];
    if (!kind_has_means(D.kind)) return fail(ctx, NS_ERR_ARG, "this likelihood kind has no means");
    const int K = D.n_comp;
    if (cap < (long)K * D.d) return fail(ctx, NS_ERR_CAPACITY, "ns_grad_logz: cap < n_comp * d");
    RunState S;
    CU(cudaMemcpyAsync(&S, ctx->state_dev + run, sizeof S, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (!S.final_done) return fail(ctx, NS_ERR_NOT_DONE, "run has not finished");
    const int nb = 304;
    const int len = K * D.d;
    ns_status es = ensure_scratch(ctx, (size_t)(nb + 1) * len);
    if (es != NS_OK) return es;
    double *part = ctx->scratch, *res = ctx->scratch + (size_t)nb * len;
    int cls = -1;
    for (int i = 0; i < (int)ctx->classes.size(); ++i)
        for (int r : ctx->classes[i].runs)
            if (r == run) cls = i;
    const RunClass &rc = ctx->classes[cls];
    const size_t smem = rc.smem + sizeof(double) * (size_t)len + 64;
    CU(kind_launch(D.kind).set_smem(D.tile, smem));
    CU(kind_launch(D.kind).grad_means(D.tile, ctx->dc, run, S.logz, part, nb, smem, rc.prec_in_smem, ctx->stream));
    CU(launch_reduce_parts(part, nb, len, res, ctx->stream));
    ctx->launches += 2;
    CU(cudaMemcpyAsync(grad, res, sizeof(double) * (size_t)len, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return NS_OK;
}

// ---- state save / load: header, then the raw device arrays in a fixed order
struct SaveHeader {
    uint64_t magic;
    int n_runs;
    long fa_len, pt_len, w_len;
};

ns_status ns_state_save(const ns_ctx *cctx, void *buf, size_t cap, size_t *n)
{
    ns_ctx *ctx = const_cast<ns_ctx *>(cctx);
    if (!ctx || !n) return NS_ERR_ARG;
    std::vector<RunState> st;
    ns_status s = read_states(ctx, st);
    if (s != NS_OK) return s;
    size_t need = sizeof(SaveHeader) + sizeof(RunState) * ctx->n_runs + sizeof(Stats) * ctx->n_runs +
                  sizeof(float) * ctx->fa_len + (sizeof(float) + 2 * sizeof(int)) * ctx->pt_len;
    for (int r = 0; r < ctx->n_runs; ++r) {
        const long nd = st[r].n_dead;
        need += sizeof(long) + (size_t)nd * (sizeof(float) * ctx->desc[r].d_pad + sizeof(float) + sizeof(double) + sizeof(int));
    }
    *n = need;
    if (!buf) return NS_OK;
    if (cap < need) return fail(ctx, NS_ERR_CAPACITY, "ns_state_save: buffer too small");
    char *p = static_cast<char *>(buf);
    SaveHeader h{0x474753535441ull, ctx->n_runs, ctx->fa_len, ctx->pt_len, ctx->w_len};
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    auto d2h = [&](const void *src, size_t bytes) -> ns_status {
        CU(cudaMemcpyAsync(p, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        p += bytes;
        return NS_OK;
    };
    if ((s = d2h(ctx->state_dev, sizeof(RunState) * ctx->n_runs)) != NS_OK) return s;
    if ((s = d2h(ctx->stats_dev, sizeof(Stats) * ctx->n_runs)) != NS_OK) return s;
    if ((s = d2h(ctx->fa, sizeof(float) * ctx->fa_len)) != NS_OK) return s;
    if ((s = d2h(ctx->logl, sizeof(float) * ctx->pt_len)) != NS_OK) return s;
    if ((s = d2h(ctx->label, sizeof(int) * ctx->pt_len)) != NS_OK) return s;
    if ((s = d2h(ctx->order, sizeof(int) * ctx->pt_len)) != NS_OK) return s;
    for (int r = 0; r < ctx->n_runs; ++r) {
        const long nd = st[r].n_dead;
        memcpy(p, &nd, sizeof nd);
        p += sizeof nd;
        const RunDesc &D = ctx->desc[r];
        if ((s = d2h(D.dead_x, sizeof(float) * (size_t)nd * D.d_pad)) != NS_OK) return s;
        if ((s = d2h(D.dead_logl, sizeof(float) * (size_t)nd)) != NS_OK) return s;
        if ((s = d2h(D.dead_logw, sizeof(double) * (size_t)nd)) != NS_OK) return s;
        if ((s = d2h(D.dead_label, sizeof(int) * (size_t)nd)) != NS_OK) return s;
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return NS_OK;
}

ns_status ns_state_load(ns_ctx *ctx, const void *buf, size_t n)
{
    if (!ctx || !buf || n < sizeof(SaveHeader)) return NS_ERR_ARG;
    const char *base = static_cast<const char *>(buf);
    SaveHeader h;
    memcpy(&h, base, sizeof h);
    if (h.magic != 0x474753535441ull || h.n_runs != ctx->n_runs || h.fa_len != ctx->fa_len || h.pt_len != ctx->pt_len ||
        h.w_len != ctx->w_len)
        return fail(ctx, NS_ERR_ARG, "ns_state_load: state does not match this context");
    // Parse and check the whole buffer on the host before anything reaches the device:
    // on any error the context keeps its previous state.
    const int R = ctx->n_runs;
    size_t off = sizeof h;
    const size_t off_state = off;
    off += sizeof(RunState) * R;
    const size_t off_stats = off;
    off += sizeof(Stats) * R;
    const size_t off_fa = off;
    off += sizeof(float) * ctx->fa_len;
    const size_t off_pt = off;
    off += (sizeof(float) + 2 * sizeof(int)) * ctx->pt_len;
    if (off > n) return fail(ctx, NS_ERR_ARG, "ns_state_load: truncated state");
    std::vector<RunState> st(R);
    memcpy(st.data(), base + off_state, sizeof(RunState) * R);
    std::vector<size_t> off_dead(R);
    std::vector<long> nds(R);
    for (int r = 0; r < R; ++r) {
        long nd;
        if (off + sizeof nd > n) return fail(ctx, NS_ERR_ARG, "ns_state_load: truncated state");
        memcpy(&nd, base + off, sizeof nd);
        off += sizeof nd;
        const RunDesc &D = ctx->desc[r];
        const size_t row = sizeof(float) * D.d_pad + sizeof(float) + sizeof(double) + sizeof(int);
        if (nd < 0 || (size_t)nd > (n - off) / row) return fail(ctx, NS_ERR_ARG, "ns_state_load: bad dead-point count");
        const RunState &S = st[r];
        if (S.n_dead != nd || S.dead_base < 0 || S.dead_base > nd || S.n_clusters < 0 || S.n_clusters > CMAX ||
            S.iter < 0)
            return fail(ctx, NS_ERR_ARG, "ns_state_load: run %d: inconsistent run state", r);
        nds[r] = nd;
        off_dead[r] = off;
        off += (size_t)nd * row;
    }
    if (off != n) return fail(ctx, NS_ERR_ARG, "ns_state_load: %zu bytes given, the state holds %zu", n, off);
    ns_status s;
    // room for the dead rows (and the iterations that follow) before the copies
    for (int r = 0; r < R; ++r) {
        const long need = nds[r] + ctx->desc[r].n_live + (long)GRAPH_ITERS * ctx->desc[r].k;
        if (need > ctx->desc[r].dead_cap && (s = alloc_dead(ctx, r, need)) != NS_OK) return s;
    }
    auto h2d = [&](void *dst, size_t at, size_t bytes) -> ns_status {
        CU(cudaMemcpyAsync(dst, base + at, bytes, cudaMemcpyHostToDevice, ctx->stream));
        return NS_OK;
    };
    if ((s = h2d(ctx->state_dev, off_state, sizeof(RunState) * R)) != NS_OK) return s;
    if ((s = h2d(ctx->stats_dev, off_stats, sizeof(Stats) * R)) != NS_OK) return s;
    // keep this context's parameter block layout: the float arena holds live x, walker state, parameters
    if ((s = h2d(ctx->fa, off_fa, sizeof(float) * ctx->fa_len)) != NS_OK) return s;
    size_t o = off_pt;
    if ((s = h2d(ctx->logl, o, sizeof(float) * ctx->pt_len)) != NS_OK) return s;
    o += sizeof(float) * ctx->pt_len;
    if ((s = h2d(ctx->label, o, sizeof(int) * ctx->pt_len)) != NS_OK) return s;
    o += sizeof(int) * ctx->pt_len;
    if ((s = h2d(ctx->order, o, sizeof(int) * ctx->pt_len)) != NS_OK) return s;
    for (int r = 0; r < R; ++r) {
        const RunDesc &D = ctx->desc[r];
        const size_t nd = (size_t)nds[r];
        size_t q = off_dead[r];
        if ((s = h2d(D.dead_x, q, sizeof(float) * nd * D.d_pad)) != NS_OK) return s;
        q += sizeof(float) * nd * D.d_pad;
        if ((s = h2d(D.dead_logl, q, sizeof(float) * nd)) != NS_OK) return s;
        q += sizeof(float) * nd;
        if ((s = h2d(D.dead_logw, q, sizeof(double) * nd)) != NS_OK) return s;
        q += sizeof(double) * nd;
        if ((s = h2d(D.dead_label, q, sizeof(int) * nd)) != NS_OK) return s;
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return NS_OK;
}

void ns_destroy(ns_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    for (auto &g : ctx->groups) {
        if (g.graph) cudaGraphExecDestroy(g.graph);
        for (auto &rc : g.classes)
            if (rc.runs_dev) cudaFree(rc.runs_dev);
        for (int i = 0; i < GRAPH_ITERS; ++i)
            for (int j = 0; j < 2; ++j)
                if (g.ev[i][j]) cudaEventDestroy(g.ev[i][j]);
        if (g.done_ev) cudaEventDestroy(g.done_ev);
        if (g.fork_ev) cudaEventDestroy(g.fork_ev);
        if (g.join_ev) cudaEventDestroy(g.join_ev);
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.ev_stream) cudaStreamDestroy(g.ev_stream);
        if (g.nz_stream) cudaStreamDestroy(g.nz_stream);
        if (g.nz_fork_ev) cudaEventDestroy(g.nz_fork_ev);
        if (g.nz_join_ev) cudaEventDestroy(g.nz_join_ev);
        if (g.pick_ev) cudaEventDestroy(g.pick_ev);
        if (g.tail_ev) cudaEventDestroy(g.tail_ev);
    }
    if (ctx->start_ev) cudaEventDestroy(ctx->start_ev);
    for (auto &rc : ctx->classes)
        if (rc.runs_dev) cudaFree(rc.runs_dev);
    for (auto &d : ctx->dead) {
        if (d.x) cudaFree(d.x);
        if (d.logl) cudaFree(d.logl);
        if (d.logw) cudaFree(d.logw);
        if (d.label) cudaFree(d.label);
    }
    void *ptrs[] = {ctx->desc_dev, ctx->state_dev, ctx->stats_dev, ctx->fa,         ctx->logl,      ctx->label,
                    ctx->order,    ctx->nbr,       ctx->lastkey,   ctx->start_slot, ctx->new_label, ctx->wint,
                    ctx->wres};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < GRAPH_ITERS; ++i)
        for (int j = 0; j < 2; ++j)
            if (ctx->ev[i][j]) cudaEventDestroy(ctx->ev[i][j]);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->rec.meta) cudaFree(ctx->rec.meta);
    if (ctx->rec.ll) cudaFree(ctx->rec.ll);
    if (ctx->rec.x) cudaFree(ctx->rec.x);
    if (ctx->rec.nz) cudaFree(ctx->rec.nz);
    if (ctx->rec.nsp) cudaFree(ctx->rec.nsp);
    if (ctx->rec_base_dev) cudaFree(ctx->rec_base_dev);
    if (ctx->graph_stream) cudaStreamDestroy(ctx->graph_stream);
    delete ctx;
}

// ------------------------------------------------------------------------
// Component entry points
// ------------------------------------------------------------------------
ns_status ns_philox(const uint32_t *ctr_dev, uint32_t key0, uint32_t key1, uint32_t *out_dev, long n, void *stream)
{
    ns_ctx *ctx = nullptr;
    if (n < 0 || (n > 0 && (!ctr_dev || !out_dev))) return NS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CU(launch_philox(ctr_dev, key0, key1, out_dev, n, s));
    CU(cudaStreamSynchronize(s));
    return NS_OK;
}

static ns_status lik_points(const ns_ctx *cctx, const float *x, long n, int mode, float *logl, float *grad,
                            const float *gout, float *gmu, void *stream)
{
    ns_ctx *ctx = const_cast<ns_ctx *>(cctx);
    if (!ctx || n < 0 || (n > 0 && !x)) return NS_ERR_ARG;
    if (n == 0) return NS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const RunDesc &D = ctx->desc[0];
    int cls = 0;
    for (int i = 0; i < (int)ctx->classes.size(); ++i)
        for (int r : ctx->classes[i].runs)
            if (r == 0) cls = i;
    const RunClass &rc = ctx->classes[cls];
    if (gmu) CU(cudaMemsetAsync(gmu, 0, sizeof(float) * (size_t)D.n_comp * D.d, s));
    CU(kind_launch(D.kind).lik_points(D.tile, ctx->dc, 0, x, n, mode, logl, grad, gout, gmu, rc.smem, rc.prec_in_smem, s));
    CU(cudaStreamSynchronize(s));
    return NS_OK;
}

ns_status ns_set_means(ns_ctx *ctx, int run, const double *means_host)
{
    if (!ctx || !means_host || run < 0 || run >= ctx->n_runs) return NS_ERR_ARG;
    const RunDesc &D = ctx->desc[run];
    if (!kind_has_means(D.kind)) return fail(ctx, NS_ERR_ARG, "this likelihood kind has no means");
    const int K = D.n_comp, d = D.d, dp = D.d_pad;
    const ParLayout L = par_layout(d, dp, K, D.kind);
    std::vector<float> m((size_t)K * dp, 0.f);
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < d; ++i) m[(size_t)k * dp + i] = (float)means_host[(size_t)k * d + i];
    CU(cudaMemcpyAsync(ctx->fa + D.par_off + L.means, m.data(), sizeof(float) * m.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    std::vector<float> pm;
    if (D.kind == NS_LIK_DENSE_MIX) {
        // P mu_k in FP64 from the master precision, as at creation
        const std::vector<double> &P = ctx->prec64[run];
        pm.assign((size_t)K * dp, 0.f);
        for (int k = 0; k < K; ++k)
            for (int i = 0; i < d; ++i) {
                double acc = 0.0;
                for (int j = 0; j < d; ++j) acc += P[(size_t)i * d + j] * means_host[(size_t)k * d + j];
                pm[(size_t)k * dp + i] = (float)acc;
            }
        CU(cudaMemcpyAsync(ctx->fa + D.par_off + L.pmu, pm.data(), sizeof(float) * pm.size(), cudaMemcpyHostToDevice,
                           ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return NS_OK;
}

ns_status ns_lik_forward(const ns_ctx *ctx, const float *x_dev, long n, float *logl_dev, float *grad_dev, void *stream)
{
    if (!logl_dev) return NS_ERR_ARG;
    return lik_points(ctx, x_dev, n, 0, logl_dev, grad_dev, nullptr, nullptr, stream);
}

ns_status ns_lik_backward(const ns_ctx *ctx, const float *x_dev, long n, const float *gout_dev, float *gx_dev,
                          float *gmu_dev, void *stream)
{
    if (!gout_dev) return NS_ERR_ARG;
    if (ctx && !kind_has_means(ctx->desc[0].kind) && gmu_dev) return NS_ERR_ARG;
    return lik_points(ctx, x_dev, n, 1, nullptr, gx_dev, gout_dev, gmu_dev, stream);
}

ns_status ns_hss(const ns_ctx *cctx, const float *x0_dev, const float *logl0_dev, long n, float lstar, double dt,
                 uint32_t iter, float *x_out_dev, float *logl_out_dev, int *steps_dev, long *stats_host, void *stream)
{
    ns_ctx *ctx = const_cast<ns_ctx *>(cctx);
    if (!ctx || n < 1 || n > NLIVE_MAX / 2 || !x0_dev || !logl0_dev || !x_out_dev || !logl_out_dev) return NS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // a private one-run view: slots [0, n) hold the start points, [n, 2n) receive the outputs
    RunDesc D = ctx->desc[0];
    const int dp = D.d_pad, d = D.d;
    const ParLayout L = par_layout(D.d, D.d_pad, D.n_comp, D.kind);
    D.n_live = (int)(2 * n);
    D.k = (int)n;
    D.x_off = 0;
    D.ws_off = (long)2 * n * dp;
    D.par_off = D.ws_off + (long)n * 3 * dp;
    D.pt_off = 0;
    D.w_off = 0;
    D.nbr_off = 0;
    D.dead_off = 0;
    D.dead_cap = n;
    const long fa_len = D.par_off + L.total;
    float *fa = nullptr, *logl = nullptr, *wres = nullptr, *dx = nullptr, *dl = nullptr;
    int *order = nullptr, *start = nullptr, *nlab = nullptr, *wint = nullptr, *lab = nullptr, *dlab = nullptr, *runs = nullptr;
    double *dw = nullptr;
    RunDesc *ddesc = nullptr;
    RunState *dstate = nullptr;
    RecView R{};
    long *rbase = nullptr;
    // every scratch buffer of this call is freed when it returns, on every path
    struct FreeAtExit {
        std::vector<void **> slots;
        ~FreeAtExit()
        {
            for (void **q : slots)
                if (*q) cudaFree(*q);
        }
    } scratch;
    scratch.slots = {(void **)&fa,    (void **)&logl,  (void **)&lab,    (void **)&order,  (void **)&start,
                     (void **)&nlab,  (void **)&wint,  (void **)&wres,   (void **)&dx,     (void **)&dl,
                     (void **)&dw,    (void **)&dlab,  (void **)&runs,   (void **)&ddesc,  (void **)&dstate,
                     (void **)&R.meta, (void **)&R.ll, (void **)&R.x,    (void **)&rbase};
    CU(cudaMalloc(&fa, sizeof(float) * fa_len));
    CU(cudaMalloc(&logl, sizeof(float) * 2 * n));
    CU(cudaMalloc(&lab, sizeof(int) * 2 * n));
    CU(cudaMalloc(&order, sizeof(int) * 2 * n));
    CU(cudaMalloc(&start, sizeof(int) * n));
    CU(cudaMalloc(&nlab, sizeof(int) * n));
    CU(cudaMalloc(&wint, sizeof(int) * WINT * n));
    CU(cudaMalloc(&wres, sizeof(float) * n));
    CU(cudaMalloc(&dx, sizeof(float) * n * dp));
    CU(cudaMalloc(&dl, sizeof(float) * n));
    CU(cudaMalloc(&dw, sizeof(double) * n));
    CU(cudaMalloc(&dlab, sizeof(int) * n));
    CU(cudaMalloc(&runs, sizeof(int)));
    CU(cudaMalloc(&ddesc, sizeof(RunDesc)));
    CU(cudaMalloc(&dstate, sizeof(RunState)));
    D.dead_x = dx;
    D.dead_logl = dl;
    D.dead_logw = dw;
    D.dead_label = dlab;
    CU(cudaMemsetAsync(fa, 0, sizeof(float) * fa_len, s));
    CU(cudaMemcpy2DAsync(fa, sizeof(float) * dp, x0_dev, sizeof(float) * d, sizeof(float) * d, n,
                         cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(fa + D.par_off, ctx->fa + ctx->desc[0].par_off, sizeof(float) * L.total, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(logl, logl0_dev, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    std::vector<int> hs(n), ho(2 * n), zero(2 * n, 0);
    for (long j = 0; j < n; ++j) {
        hs[j] = (int)j;
        ho[j] = (int)(n + j);
        ho[n + j] = (int)j;
    }
    CU(cudaMemcpyAsync(start, hs.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(order, ho.data(), sizeof(int) * 2 * n, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(nlab, zero.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(lab, zero.data(), sizeof(int) * 2 * n, cudaMemcpyHostToDevice, s));
    RunState S;
    memset(&S, 0, sizeof S);
    S.iter = (int)iter;
    S.dt = dt;
    S.lstar = lstar;
    S.n_dead = n;
    S.remain_min = S.remain_max = (int)n;
    const int zr = 0;
    CU(cudaMemcpyAsync(runs, &zr, sizeof(int), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ddesc, &D, sizeof D, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(dstate, &S, sizeof S, cudaMemcpyHostToDevice, s));
    DevCtx C{};
    C.n_runs = 1;
    C.desc = ddesc;
    C.state = dstate;
    C.stats = nullptr;
    C.fa = fa;
    C.logl = logl;
    C.label = lab;
    C.order = order;
    C.start_slot = start;
    C.new_label = nlab;
    C.wint = wint;
    C.wres_logl = wres;
    C.nbr = nullptr;
    int cls = 0;
    for (int i = 0; i < (int)ctx->classes.size(); ++i)
        for (int r : ctx->classes[i].runs)
            if (r == 0) cls = i;
    RunClass rc = ctx->classes[cls];
    // the launch form the context chose for run 0 (held by its group's copy of the class)
    for (auto &g : ctx->groups)
        for (auto &gc : g.classes)
            for (int r : gc.runs)
                if (r == 0) rc = gc;
    // the single-pass form where the context uses it and all n walkers are resident
    int single = 0;
    if (ctx->rec.rec_len > 0) {
        int per_sm = 0, n_sm = 0;
        CU(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
        CU(kind_launch(D.kind).hss1_occ(D.tile, rc.smem, &per_sm));
        const long gpc = HSS_THREADS / tile_of(D.tile).g;
        single = (n + gpc - 1) / gpc <= (long)per_sm * n_sm ? 1 : 0;
    }
    if (D.midpoint && (!single || std::min(ctx->rec.rec_len, D.n_steps) < D.n_steps))
        return fail(ctx, NS_ERR_ARG, "ns_hss: midpoint needs the single pass with records for every step");
    if (single) {
        R.rec_len = std::min(ctx->rec.rec_len, D.n_steps);
        R.xs = dp;
        const long rows = n * (long)R.rec_len;
        const long zero_base = 0;
        CU(cudaMalloc(&R.meta, sizeof(uint2) * rows));
        CU(cudaMalloc(&R.ll, sizeof(float) * rows));
        CU(cudaMalloc(&R.x, sizeof(float) * rows * dp));
        CU(cudaMalloc(&rbase, sizeof(long)));
        CU(cudaMemcpyAsync(rbase, &zero_base, sizeof(long), cudaMemcpyHostToDevice, s));
        if (rc.coop > 0)  // the context's dense form: 16 walkers per CTA sharing P (tensor cores if coop_tr = 0)
            CU(kind_launch(D.kind).hss1_coop(D.tile, C, runs, 1, (int)n, R, rbase, rc.coop_smem, rc.coop_tr, s));
        else
            CU(kind_launch(D.kind).hss1(D.tile, C, runs, 1, (int)n, R, rbase, rc.smem, rc.prec_in_smem, s));
        CU(launch_hss_pick(C, runs, 1, (int)n, R, rbase, s));
        if (D.midpoint)
            CU(kind_launch(D.kind).eval_new(D.tile, C, runs, 1, (int)n, rc.smem, rc.prec_in_smem, s));
    }
    for (int phase = 0; phase < 3; ++phase)
        CU(kind_launch(D.kind).hss(D.tile, C, runs, 1, (int)n, single ? (phase | 4) : phase, rc.smem,
                                   rc.prec_in_smem, s));
    CU(cudaMemcpy2DAsync(x_out_dev, sizeof(float) * d, fa + (long)n * dp, sizeof(float) * dp, sizeof(float) * d, n,
                         cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(logl_out_dev, logl + n, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(&S, dstate, sizeof S, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (steps_dev) {
        std::vector<int> st(n, S.t_stop);
        CU(cudaMemcpy(steps_dev, st.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    }
    if (stats_host) {
        stats_host[0] = S.n_in;
        stats_host[1] = S.n_out;
        stats_host[2] = S.t_save;
        stats_host[3] = S.t_stop;
        stats_host[4] = S.n_fold;
    }
    return NS_OK;
}

ns_status ns_knn_components(const float *x_dev, int m, int d, int *comp_dev, int *n_comp_host, void *stream)
{
    ns_ctx *ctx = nullptr;
    if (m < 1 || m > NLIVE_MAX || d < 1 || d > DMAX || !x_dev || !comp_dev) return NS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevScratch label, csize, nbr, nc, lk;
    CU(cudaMalloc(&label.p, sizeof(int) * m));
    CU(cudaMalloc(&csize.p, sizeof(int) * CMAX));
    CU(cudaMalloc(&nbr.p, sizeof(int) * (size_t)m * KNN_K));
    CU(cudaMalloc(&nc.p, sizeof(int)));
    CU(cudaMalloc(&lk.p, sizeof(unsigned long long) * m));
    std::vector<int> cs(CMAX, 0);
    cs[0] = m;
    CU(cudaMemsetAsync(label.p, 0, sizeof(int) * m, s));
    CU(cudaMemcpyAsync(csize.p, cs.data(), sizeof(int) * CMAX, cudaMemcpyHostToDevice, s));
    CU(launch_knn_components(x_dev, m, d, label.as<int>(), csize.as<int>(), nbr.as<int>(), comp_dev,
                             lk.as<unsigned long long>(), nc.as<int>(), s));
    int h = 0;
    CU(cudaMemcpyAsync(&h, nc.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (n_comp_host) *n_comp_host = h;
    return NS_OK;
}

ns_status ns_territory(const float *surv_dev, const int *surv_label_dev, int m_s, const float *xn_dev,
                       const int *want_dev, int k, int d, int *keep_dev, void *stream)
{
    ns_ctx *ctx = nullptr;
    if (m_s < 0 || m_s > NLIVE_MAX || k < 0 || k > NLIVE_MAX || d < 1 || d > DMAX || (m_s > 0 && (!surv_dev || !surv_label_dev)) ||
        (k > 0 && (!xn_dev || !want_dev || !keep_dev)))
        return NS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CU(launch_territory_plain(surv_dev, surv_label_dev, m_s, xn_dev, want_dev, k, d, keep_dev, s));
    CU(cudaStreamSynchronize(s));
    return NS_OK;
}

ns_status ns_sort_logl(const float *logl_dev, int n, int *order_dev, void *stream)
{
    ns_ctx *ctx = nullptr;
    if (n < 1 || n > NLIVE_MAX || !logl_dev || !order_dev) return NS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CU(launch_sort_logl(logl_dev, n, order_dev, s));
    CU(cudaStreamSynchronize(s));
    return NS_OK;
}

ns_status ns_stats_update(int n_clusters, const int *counts, const double *logx0, const double *logzx0,
                          const double *logxx0, int k, const int *labels, const double *logl, double *out)
{
    ns_ctx *ctx = nullptr;
    if (n_clusters < 1 || n_clusters > CMAX || k < 1 || !counts || !logx0 || !labels || !logl || !out) return NS_ERR_ARG;
    Stats T;
    for (int c = 0; c < CMAX; ++c) {
        T.logZp[c] = T.logZp2[c] = T.logZXp[c] = T.logZpXp[c] = T.logXp[c] = T.logXp2[c] = -INFINITY;
        T.n[c] = 0;
        T.alive[c] = 0;
    }
    for (int i = 0; i < CMAX * CMAX; ++i) T.logXX[i] = -INFINITY;
    std::vector<int> left(n_clusters);
    for (int c = 0; c < n_clusters; ++c) {
        T.alive[c] = counts[c] > 0;
        T.n[c] = counts[c];
        T.logXp[c] = logx0[c];
        T.logXp2[c] = 2.0 * logx0[c];
        T.logZXp[c] = logzx0 ? logzx0[c] : -INFINITY;
        for (int q = 0; q < n_clusters; ++q)
            if (q != c && logxx0) T.logXX[c * CMAX + q] = logxx0[(size_t)c * n_clusters + q];
        left[c] = counts[c];
    }
    for (int j = 0; j < k; ++j) {
        if (labels[j] < 0 || labels[j] >= n_clusters || --left[labels[j]] < 0)
            return fail(nullptr, NS_ERR_ARG, "ns_stats_update: more kills than live points in a cluster");
    }
    DevScratch dst, zz, kL, kP, lw;
    CU(cudaMalloc(&dst.p, sizeof(Stats)));
    CU(cudaMalloc(&zz.p, 2 * sizeof(double)));
    CU(cudaMalloc(&kL.p, sizeof(double) * k));
    CU(cudaMalloc(&kP.p, sizeof(int) * k));
    CU(cudaMalloc(&lw.p, sizeof(double) * k));
    const double z0[2] = {-INFINITY, -INFINITY};
    CU(cudaMemcpy(dst.p, &T, sizeof T, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(zz.p, z0, sizeof z0, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(kL.p, logl, sizeof(double) * k, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(kP.p, labels, sizeof(int) * k, cudaMemcpyHostToDevice));
    CU(launch_stats_plain(dst.as<Stats>(), zz.as<double>(), k, kL.as<double>(), kP.as<int>(), lw.as<double>(),
                          nullptr));
    CU(cudaDeviceSynchronize());
    Stats R;
    double zr[2];
    CU(cudaMemcpy(&R, dst.p, sizeof R, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(zr, zz.p, sizeof zr, cudaMemcpyDeviceToHost));
    out[0] = zr[0];
    out[1] = zr[1];
    out[2] = 0.0;
    for (int c = 0; c < n_clusters; ++c) {
        out[3 + 3 * c] = R.logXp[c];
        out[3 + 3 * c + 1] = R.logXp2[c];
        out[3 + 3 * c + 2] = R.logZXp[c];
    }
    CU(cudaMemcpy(out + 3 + 3 * n_clusters, lw.p, sizeof(double) * k, cudaMemcpyDeviceToHost));
    return NS_OK;
}

}  // extern "C"
