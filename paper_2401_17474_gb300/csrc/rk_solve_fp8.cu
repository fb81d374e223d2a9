// rk_solve_fp8.cu -- FP8-row instantiations of the persistent RKAB kernel.
#include "rk_solve_kernel.cuh"

namespace rk {

#define V_(NT, VPT, KA, W) SolveVariant{NT, VPT, KA, W, rkab_kernel<NT, VPT, ELT_FP8, KA, W>, 1, false}
#define VJ_(NT, VPT, KA) SolveVariant{NT, VPT, KA, 1, rkab_kernel<NT, VPT, ELT_FP8, KA, 1, 1, true>, 1, true}
#define V2_(NT, VPT) SolveVariant{NT, VPT, false, 1, rkab_kernel<NT, VPT, ELT_FP8, false, 1, 2>, 2, false}
#define VX_(NT, VPT) SolveVariant{NT, VPT, true, 1, rkab_kernel<NT, VPT, ELT_FP8, true, 1, 1, false, true>, 1, false, true}
static const SolveVariant kTab[] = {
    V_(32, 1, true, 1),    V_(32, 2, true, 1),    V_(32, 4, true, 1),
    V_(128, 2, true, 1),   V_(128, 3, true, 1),   V_(128, 5, true, 1),
    V_(256, 3, true, 1),   V_(256, 4, true, 1),   V_(256, 5, true, 1),   V_(256, 6, true, 1),
    V_(256, 8, true, 1),   V_(256, 10, true, 1),
    V_(512, 6, false, 1),  V_(512, 8, false, 1),  V_(512, 10, false, 1),
    V_(128, 2, false, 2),  V_(128, 3, false, 2),  V_(128, 5, false, 2),
    V_(256, 3, false, 2),  V_(256, 4, false, 2),  V_(256, 5, false, 2),  V_(256, 6, false, 2),
    V_(256, 8, false, 2),  V_(256, 10, false, 2),
    V_(128, 2, false, 4),  V_(128, 3, false, 4),  V_(128, 5, false, 4),
    V_(256, 3, false, 4),  V_(256, 4, false, 4),  V_(256, 5, false, 4),  V_(256, 6, false, 4),
    V_(256, 8, false, 4),
    V2_(128, 2), V2_(128, 5), V2_(256, 5), V2_(256, 8), V2_(256, 10),
    VJ_(32, 1, true),   VJ_(32, 2, true),   VJ_(32, 4, true),
    VJ_(128, 2, true),  VJ_(128, 3, true),  VJ_(128, 5, true),
    VJ_(256, 3, true),  VJ_(256, 4, true),  VJ_(256, 5, true),  VJ_(256, 6, true),
    VJ_(256, 8, true),  VJ_(256, 10, true),
    VJ_(512, 6, false), VJ_(512, 8, false), VJ_(512, 10, false),
    VX_(256, 12), VX_(256, 16),
};
#undef V_
#undef V2_
#undef VX_
#undef VJ_

const SolveVariant* solve_variants_fp8(int* count) {
    *count = (int)(sizeof(kTab) / sizeof(kTab[0]));
    return kTab;
}

}  // namespace rk
