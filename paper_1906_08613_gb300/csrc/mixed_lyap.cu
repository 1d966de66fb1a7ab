// Instantiations of the mixed-precision Lyapunov kernels (see mixed_solver.cuh).
#include "mixed_warp.cuh"

namespace ss {

// cfg -> (B, T, residual) per precision; the table is mirrored in mixed_api.cu.
cudaError_t launch_mixed_trlyap(int prec, int cfg, const Operands &o, const Sched &s, const Launch &l,
                             cudaStream_t st, int raw)
{
    using namespace mx;
    if (prec == P_FP32) {
        switch (cfg) {
        case 0: return launch_mixed_syl<16, 64, true, P_FP32, R_DF>(o, s, l, st, raw);
        case 1: return launch_mixed_syl<16, 128, true, P_FP32, R_DF>(o, s, l, st, raw);
        case 2: return launch_mixed_syl<32, 128, true, P_FP32, R_DF>(o, s, l, st, raw);
        case 3: return launch_mixed_syl<16, 128, true, P_FP32, R_FP64>(o, s, l, st, raw);
        case 4: return launch_mixed_syl<32, 128, true, P_FP32, R_FP64>(o, s, l, st, raw);
        case 5: return wb::launch_warp_syl<4, true>(o, s, l, st, raw);
        case 6: return wb::launch_warp_syl<2, true>(o, s, l, st, raw);
        case 7: return wb::launch_warp_syl<8, true>(o, s, l, st, raw);
        }
    } else if (prec == P_TF32) {
        switch (cfg) {
        case 0: return launch_mixed_syl<16, 64, true, P_TF32, R_DF>(o, s, l, st, raw);
        case 1: return launch_mixed_syl<32, 128, true, P_TF32, R_DF>(o, s, l, st, raw);
        case 2: return launch_mixed_syl<16, 64, true, P_TF32, R_FP64>(o, s, l, st, raw);
        case 3: return launch_mixed_syl<32, 128, true, P_TF32, R_FP64>(o, s, l, st, raw);
        case 4: return wb::launch_warp_tc<true, P_TF32>(o, s, l, st, raw);
        }
    } else if (prec == P_BF16) {
        switch (cfg) {
        case 0: return launch_mixed_syl<16, 64, true, P_BF16, R_DF>(o, s, l, st, raw);
        case 1: return launch_mixed_syl<32, 128, true, P_BF16, R_DF>(o, s, l, st, raw);
        case 2: return launch_mixed_syl<16, 64, true, P_BF16, R_FP64>(o, s, l, st, raw);
        case 3: return launch_mixed_syl<32, 128, true, P_BF16, R_FP64>(o, s, l, st, raw);
        case 4: return wb::launch_warp_tc<true, P_BF16>(o, s, l, st, raw);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace ss
