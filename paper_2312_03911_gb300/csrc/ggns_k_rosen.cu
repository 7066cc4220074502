// ggns_k_rosen.cu -- walker-layout kernels for likelihood kind NS_LIK_ROSENBROCK.
#define GGNS_KIND NS_LIK_ROSENBROCK
#define GGNS_KIND_NS kind_rosen
#include "ggns_kind_impl.cuh"

namespace ggns {
const KindLaunch &kind_launch_rosen()
{
    static const KindLaunch L{kind_rosen::prior, kind_rosen::hss, kind_rosen::lik, kind_rosen::grad, kind_rosen::smem_attr, kind_rosen::hss1,
                                kind_rosen::hss1_occ, kind_rosen::hss1_coop,
                                kind_rosen::hss1_coop_occ, kind_rosen::eval_new};
    return L;
}
}  // namespace ggns
