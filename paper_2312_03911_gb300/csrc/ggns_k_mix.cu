// ggns_k_mix.cu -- walker-layout kernels for likelihood kind NS_LIK_MIX_ISO.
#define GGNS_KIND NS_LIK_MIX_ISO
#define GGNS_KIND_NS kind_mix
#include "ggns_kind_impl.cuh"

namespace ggns {
const KindLaunch &kind_launch_mix()
{
    static const KindLaunch L{kind_mix::prior, kind_mix::hss, kind_mix::lik, kind_mix::grad, kind_mix::smem_attr, kind_mix::hss1,
                                kind_mix::hss1_occ, kind_mix::hss1_coop,
                                kind_mix::hss1_coop_occ, kind_mix::eval_new};
    return L;
}
}  // namespace ggns
