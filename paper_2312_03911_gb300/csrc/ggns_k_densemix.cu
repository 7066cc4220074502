// ggns_k_densemix.cu -- walker-layout kernels for likelihood kind NS_LIK_DENSE_MIX.
#define GGNS_KIND NS_LIK_DENSE_MIX
#define GGNS_KIND_NS kind_densemix
#include "ggns_kind_impl.cuh"

namespace ggns {
const KindLaunch &kind_launch_densemix()
{
    static const KindLaunch L{kind_densemix::prior, kind_densemix::hss, kind_densemix::lik, kind_densemix::grad, kind_densemix::smem_attr, kind_densemix::hss1,
                                kind_densemix::hss1_occ, kind_densemix::hss1_coop,
                                kind_densemix::hss1_coop_occ, kind_densemix::eval_new};
    return L;
}
}  // namespace ggns
