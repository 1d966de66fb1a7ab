// Configuration tables and dispatch of the mixed-precision modes.
#include "ss_internal.h"

namespace ss {

cudaError_t launch_mixed_trsyl(int prec, int cfg, const Operands &o, const Sched &s, const Launch &l,
                               cudaStream_t st, int raw);
cudaError_t launch_mixed_trlyap(int prec, int cfg, const Operands &o, const Sched &s, const Launch &l,
                                cudaStream_t st, int raw);
cudaError_t launch_mixed_potrf(int prec, int cfg, const Operands &o, const Sched &s, const Launch &l,
                               cudaStream_t st, int raw);

namespace {

// variant: bit 0 = residual (0 double-float on the FP32 pipe, 1 FP64 FMA);
// bit 1 = solve (0 blocked lazy with block size `block`; 1 warp-block
// wavefront, 32 x 32 blocks, one warp per block of a block anti-diagonal).
const Config kFp32Cfg[] = {{16, 64, 0},  {16, 128, 0}, {32, 128, 0}, {16, 128, 1},
                           {32, 128, 1}, {32, 128, 2}, {32, 64, 2},  {32, 256, 2}};
// variant bit 2: the right-hand side resident in tensor memory, trailing
// updates by tcgen05 MMA (n > 128 falls back to the warp-block wavefront).
const Config kTcCfg[] = {{16, 64, 0}, {32, 128, 0}, {16, 64, 1}, {32, 128, 1}, {32, 128, 4}};
// Cholesky (blocked lazy factorization, then factor refinement).
const Config kCholFp32Cfg[] = {{16, 64, 0}, {16, 128, 0}, {32, 128, 0}, {32, 128, 1}};
// variant bit 2: the trailing matrix resident in tensor memory, SYRK updates
// by tcgen05 MMA (TF32 / BF16 only; n > 256 falls back to the blocked path).
const Config kCholTcCfg[] = {{16, 64, 0}, {32, 128, 0}, {32, 128, 1}, {32, 128, 4}};

// Low-precision arithmetic of a mode: 0 FP32, 1 TF32, 2 BF16; -1 not mixed.
int mode_prec(int mode)
{
    switch (mode) {
    case SS_MODE_FP32_REFINED: case SS_MODE_FP32_RAW: return 0;
    case SS_MODE_TF32_REFINED: case SS_MODE_TF32_RAW: return 1;
    case SS_MODE_BF16_REFINED: case SS_MODE_BF16_RAW: return 2;
    }
    return -1;
}
bool mode_raw(int mode)
{
    return mode == SS_MODE_FP32_RAW || mode == SS_MODE_TF32_RAW || mode == SS_MODE_BF16_RAW;
}

}  // namespace

int mixed_config_count(int op, int mode)
{
    const int p = mode_prec(mode);
    if (p < 0) return 0;
    if (op == SS_OP_POTRF)
        return p == 0 ? (int)(sizeof(kCholFp32Cfg) / sizeof(Config)) : (int)(sizeof(kCholTcCfg) / sizeof(Config));
    return p == 0 ? (int)(sizeof(kFp32Cfg) / sizeof(Config)) : (int)(sizeof(kTcCfg) / sizeof(Config));
}

const Config *mixed_config_get(int op, int mode, int cfg)
{
    if (cfg < 0 || cfg >= mixed_config_count(op, mode)) return nullptr;
    if (op == SS_OP_POTRF) return mode_prec(mode) == 0 ? &kCholFp32Cfg[cfg] : &kCholTcCfg[cfg];
    return mode_prec(mode) == 0 ? &kFp32Cfg[cfg] : &kTcCfg[cfg];
}

// Scratch per instance in floats per n^2: the right-hand side / correction
// and the reciprocal divisors; the warp-block and tensor-memory variants
// (Sylvester / Lyapunov) also keep FP32 copies of L and U.
long long mixed_scratch_per_n2(int op, int mode)
{
    if (mixed_config_count(op, mode) <= 0) return 0;
    return op != SS_OP_POTRF ? 4 : 2;
}

// Kernels one launch group of (op, mode, cfg) launches: the tensor-memory
// Cholesky factors in one pass and refines in a second.
int mixed_launches(int op, int mode, int cfg)
{
    const Config *c = mixed_config_get(op, mode, cfg);
    return (c && op == SS_OP_POTRF && (c->variant & 4)) ? 2 : 1;
}

cudaError_t launch_mixed(int op, const Operands &o, const Sched &s, const Launch &l, cudaStream_t st)
{
    const int p = mode_prec(l.mode);
    const int raw = mode_raw(l.mode) ? 1 : 0;
    if (op == SS_OP_TRSYL) return launch_mixed_trsyl(p, l.cfg, o, s, l, st, raw);
    if (op == SS_OP_TRLYAP) return launch_mixed_trlyap(p, l.cfg, o, s, l, st, raw);
    if (op == SS_OP_POTRF) return launch_mixed_potrf(p, l.cfg, o, s, l, st, raw);
    return cudaErrorNotSupported;
}

}  // namespace ss
