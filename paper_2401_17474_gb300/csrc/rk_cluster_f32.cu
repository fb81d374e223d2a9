// rk_cluster_f32.cu -- F32-row instantiations of the cluster RKAB kernel.
#include "rk_cluster_kernel.cuh"

namespace rk {

#define V_(NT, VPT, W) ClusterVariant{NT, VPT, W, rkab_cluster_kernel<NT, VPT, ELT_F32, W>}
static const ClusterVariant kTab[] = {
    V_(128, 2, 4), V_(128, 3, 4), V_(128, 5, 4), V_(128, 8, 4),
    V_(128, 2, 6), V_(128, 3, 6), V_(128, 5, 6), V_(128, 8, 6),
    V_(256, 6, 2), V_(256, 9, 2), V_(256, 13, 2),
};
#undef V_

const ClusterVariant* cluster_variants_f32(int* count) {
    *count = (int)(sizeof(kTab) / sizeof(kTab[0]));
    return kTab;
}

}  // namespace rk
