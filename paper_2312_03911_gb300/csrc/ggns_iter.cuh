// ggns_iter.cuh -- host-side launchers of the libggns kernels (internal).
#pragma once

#include "ggns_internal.cuh"

namespace ggns {

// walker tiles: id -> (lanes per walker, components per lane)
constexpr int N_TILES = 15;
__host__ __device__ inline Tile tile_of(int id)
{
    constexpr int g[N_TILES] = {1, 1, 2, 4, 8, 16, 32, 32, 32, 4, 16, 8, 16, 32, 32};
    constexpr int e[N_TILES] = {2, 4, 4, 4, 4, 4, 4, 8, 16, 8, 2, 8, 8, 1, 2};
    return Tile{g[id], e[id]};
}

size_t select_smem_bytes(int n_live_max);
size_t sort_smem_bytes(int n_live_max);
size_t knn_smem_bytes(int d);
size_t cluster_smem_bytes(int n_live_max);
size_t evscratch_bytes();

cudaError_t prepare_iteration_kernels(size_t sel_smem, size_t knn_smem, size_t cl_smem, size_t sort_smem);
// run-range launchers: runs r0 .. r0 + n_runs - 1
cudaError_t launch_evidence(const DevCtx &C, int r0, int n_runs, size_t smem, cudaStream_t s);
cudaError_t launch_final(const DevCtx &C, int r0, int n_runs, size_t smem, cudaStream_t s);
cudaError_t launch_noise(const DevCtx &C, const int *runs, int nr, int blocks_per_run, const RecView &R,
                         const long *rec_base, cudaStream_t s);
cudaError_t launch_hss_pick(const DevCtx &C, const int *runs, int nr, int max_k, const RecView &R,
                            const long *rec_base, cudaStream_t s);
cudaError_t launch_term(const DevCtx &C, int r0, int n_runs, cudaStream_t s);
cudaError_t launch_territory(const DevCtx &C, int r0, int n_runs, int max_k, int max_d, cudaStream_t s);
cudaError_t launch_territory_plain(const float *surv, const int *surv_label, int m_s, const float *xn, const int *want,
                                   int k, int d, int *keep, cudaStream_t s);
cudaError_t launch_term_cluster_sort(const DevCtx &C, int r0, int n_runs, unsigned long long *lastkey, size_t smem,
                                     bool do_term, bool clustering, cudaStream_t s);
cudaError_t launch_tail(const DevCtx &C, int r0, int n_runs, cudaStream_t s);
cudaError_t launch_knn(const DevCtx &C, int r0, int n_runs, int max_nlive, size_t smem, cudaStream_t s);
cudaError_t launch_info(const DevCtx &C, int r, double logz, double *out, cudaStream_t s);
cudaError_t launch_export(const DevCtx &C, int r, int d, int d_pad, double logz, double *x, double *logp, long n,
                          cudaStream_t s);
cudaError_t launch_reduce_parts(const double *part, int n_parts, int len, double *out, cudaStream_t s);

cudaError_t launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, long n, cudaStream_t s);
cudaError_t launch_sort_logl(const float *logl, int n, int *order, cudaStream_t s);
cudaError_t launch_knn_components(const float *x, int n, int d, const int *label, const int *csize, int *nbr,
                                  int *comp, unsigned long long *lastkey, int *ncomp, cudaStream_t s);
cudaError_t launch_stats_plain(Stats *st, double *zz, int k, const double *kL, const int *kP, double *logw,
                               cudaStream_t s);

// message returned by ns_last_error(NULL)
void set_global_error(const char *msg);

// per likelihood kind (ggns_k_<kind>.cu)
struct KindLaunch {
    cudaError_t (*prior)(int tile, const DevCtx &C, const int *runs, int nr, int max_n, size_t smem, int pis,
                         cudaStream_t s);
    cudaError_t (*hss)(int tile, const DevCtx &C, const int *runs, int nr, int max_k, int phase, size_t smem,
                       int pis, cudaStream_t s);
    cudaError_t (*lik_points)(int tile, const DevCtx &C, int run, const float *x, long n, int mode, float *logl,
                              float *grad, const float *gout, float *gmu, size_t smem, int pis, cudaStream_t s);
    cudaError_t (*grad_means)(int tile, const DevCtx &C, int run, double logz, double *part, int n_blocks,
                              size_t smem, int pis, cudaStream_t s);
    cudaError_t (*set_smem)(int tile, size_t smem);
    cudaError_t (*hss1)(int tile, const DevCtx &C, const int *runs, int nr, int max_k, const RecView &R,
                        const long *rec_base, size_t smem, int pis, cudaStream_t s);
    cudaError_t (*hss1_occ)(int tile, size_t smem, int *blocks_per_sm);
    // CTA-cooperative single pass of the dense kinds (cudaErrorInvalidValue elsewhere): tr > 0 rows
    // of P per shared-memory tile with the contraction on CUDA cores; tr = 0 on the tensor cores
    cudaError_t (*hss1_coop)(int tile, const DevCtx &C, const int *runs, int nr, int max_k, const RecView &R,
                             const long *rec_base, size_t smem, int tr, cudaStream_t s);
    cudaError_t (*hss1_coop_occ)(int tile, size_t smem, int tr, int *blocks_per_sm);
    // the reversible step (midpoint): the pick's drawn states tested against L*
    cudaError_t (*eval_new)(int tile, const DevCtx &C, const int *runs, int nr, int max_k, size_t smem, int pis,
                            cudaStream_t s);
};
const KindLaunch &kind_launch(int kind);

}  // namespace ggns
