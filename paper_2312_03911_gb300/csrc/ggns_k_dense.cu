// ggns_k_dense.cu -- walker-layout kernels for likelihood kind NS_LIK_DENSE_GAUSS.
#define GGNS_KIND NS_LIK_DENSE_GAUSS
#define GGNS_KIND_NS kind_dense
#include "ggns_kind_impl.cuh"

namespace ggns {
const KindLaunch &kind_launch_dense()
{
    static const KindLaunch L{kind_dense::prior, kind_dense::hss, kind_dense::lik, kind_dense::grad, kind_dense::smem_attr, kind_dense::hss1,
                                kind_dense::hss1_occ, kind_dense::hss1_coop,
                                kind_dense::hss1_coop_occ, kind_dense::eval_new};
    return L;
}
}  // namespace ggns
