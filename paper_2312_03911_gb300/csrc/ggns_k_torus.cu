// ggns_k_torus.cu -- walker-layout kernels for likelihood kind NS_LIK_TORUS.
#define GGNS_KIND NS_LIK_TORUS
#define GGNS_KIND_NS kind_torus
#include "ggns_kind_impl.cuh"

namespace ggns {
const KindLaunch &kind_launch_torus()
{
    static const KindLaunch L{kind_torus::prior, kind_torus::hss, kind_torus::lik, kind_torus::grad, kind_torus::smem_attr,
                                kind_torus::hss1, kind_torus::hss1_occ, kind_torus::hss1_coop,
                                kind_torus::hss1_coop_occ, kind_torus::eval_new};
    return L;
}
}  // namespace ggns
