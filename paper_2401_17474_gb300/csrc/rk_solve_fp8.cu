// rk_solve_fp8.cu -- FP8-row instantiations of the persistent RKAB kernel.
#include "rk_solve_kernel.cuh"

namespace rk {

#define V_(NT, VPT, KA, W) SolveVariant{NT, VPT, KA, W, rkab_kernel<NT, VPT, ELT_FP8, KA, W>}
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
};
#undef V_

const SolveVariant* solve_variants_fp8(int* count) {
    *count = (int)(sizeof(kTab) / sizeof(kTab[0]));
    return kTab;
}

}  // namespace rk
