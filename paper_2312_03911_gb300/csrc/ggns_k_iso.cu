// ggns_k_iso.cu -- walker-layout kernels for likelihood kind NS_LIK_ISO_GAUSS.
#define GGNS_KIND NS_LIK_ISO_GAUSS
#define GGNS_KIND_NS kind_iso
#include "ggns_kind_impl.cuh"

namespace ggns {
const KindLaunch &kind_launch_iso()
{
    static const KindLaunch L{kind_iso::prior, kind_iso::hss, kind_iso::lik, kind_iso::grad, kind_iso::smem_attr, kind_iso::hss1,
                                kind_iso::hss1_occ, kind_iso::hss1_coop,
                                kind_iso::hss1_coop_occ, kind_iso::eval_new};
    return L;
}
}  // namespace ggns
