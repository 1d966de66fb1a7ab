// Internal interfaces between the C-ABI layer (api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/smallsolve.h"

namespace ss {

// Operands of one batched call, exactly as the caller passed them.
struct Operands {
    const int *n;
    const double *const *A;   // potrf: A; trsyl/trlyap: L
    const int *lda;
    const double *const *U;   // trsyl: U
    const int *ldu;
    const double *const *C;   // trsyl: C; trlyap: S
    const int *ldc;
    double *const *X;
    const int *ldx;
    int *info;
    const int *m;             // rectangular Sylvester: rows of X (null: m = n)
};

// Device-side workspace produced by the binning pre-pass.
//   meta[META_COUNT]          number of instances with a valid size
//   meta[META_BIN_LO + k]     first position (in perm) of size bin k
//   meta[META_BIN_HI + k]     one past the last position of size bin k
//   meta[META_HEAD + g]       work-queue head of launch group g
//   meta[META_RNG + g]        nonzero if a double-float solve of group g left
//                             its range (an instance has info SS_INFO_RANGE)
//   meta[META_SCL + g]        nonzero if an instance of double-float group g
//                             needs rescaling (DfInst::pend)
//   meta[META_SCL_HEAD + g]   work-queue head of that scaled pass (for a
//                             tensor-memory Cholesky group: of its
//                             refinement pass)
//   perm[w]                   instance index at position w (sizes descending)
//   scr[w]                    element offset of position w's scratch area
constexpr int META_COUNT = 0;
constexpr int META_BIN_LO = 16;
constexpr int META_BIN_HI = 32;
constexpr int META_HEAD = 48;
constexpr int META_RANGE = 64;     // pairs (lo, hi) per launch group, 2 * MAX_GROUPS
constexpr int MAX_GROUPS = 16;
constexpr int META_RNG = 96;       // MAX_GROUPS flags
constexpr int META_SCL = 112;      // MAX_GROUPS flags
constexpr int META_SCL_HEAD = 128; // MAX_GROUPS queue heads
constexpr int META_INTS = 144;
constexpr int NUM_BINS = SS_NUM_BINS;   // bin(n) = ceil(log2(max(n,1))), n <= 4096

// Per-instance state of the double-float pipelines.  Sylvester / Lyapunov:
// for an instance out of DfScale's band, the zero-shift pass writes the
// largest biased FP64 exponents of the operator (L and U) and of the
// right-hand side, and the largest diagonal magnitude of L and U (the
// singular-divisor threshold), for the rescaled pass.  pend: set by the
// unscaled pipeline when the instance needs the rescaled one (Cholesky:
// found out of DfScale's band while the solve read A).  The binning pre-pass
// zeroes every entry.
struct DfInst {
    int eo, ec;
    int pend;
    int pad;
    unsigned long long maxdiag;   // bits of a nonnegative double
};

struct Sched {
    int *meta;
    const int *perm;
    const DfInst *dfs;         // per instance, indexed by instance (SS_MODE_DF / AUTO calls), may be null
    const long long *scr;      // scratch offsets (elements), may be null
    void *scratch;             // scratch base, may be null
    long long scratch_elems;   // capacity in elements of the scratch element type
};

// A launch over the positions [meta[META_RANGE+2g], meta[META_RANGE+2g+1]).
struct Launch {
    int group;
    int cfg;                   // index into the op's configuration table
    int mode;
    int max_n;
    int batch;
};

size_t workspace_bytes(int op, int batch, int max_n, int mode);
// The parts of a workspace of work_bytes laid out as workspace_bytes counts them.
void carve_workspace(void *d_work, size_t work_bytes, int op, int batch, int max_n, int mode, Sched *s);

// Binning pre-pass: sorts valid instances by size (descending), fills bins,
// scratch offsets and the launch-group ranges, resets the queue heads.
// group_of_bin[k] is the launch group of size bin k (-1: none, only for bins
// that cannot hold instances); ngroups groups are used.
// With d_m (rectangular Sylvester) the sort key of an instance is max(m, n),
// and m outside [0, max_m] is a bad size too.  It also zeroes s.dfs when
// present.
cudaError_t launch_binning(int batch, int max_n, const int *d_n, int *d_info, const Sched &s,
                           const int *group_of_bin, int ngroups, long long scratch_per_n2,
                           cudaStream_t st, const int *d_m = nullptr, int max_m = 0);

// Configuration tables.
struct Config {
    int block;
    int threads;
    int variant;
};
int config_count(int op, int mode);
const Config *config_get(int op, int mode, int cfg);
int config_default(int op, int mode, int max_n, int batch);

// Kernel launchers (one per op).  Return cudaSuccess or the launch error.
cudaError_t launch_potrf(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st);
cudaError_t launch_trsyl(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st);
cudaError_t launch_trlyap(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st);

// Sylvester / Lyapunov with warp-specialised CTAs (block B, nu update warps
// plus one diagonal warp); df: the update warps compute in double-float on the
// FP32 pipe (SS_MODE_DF), otherwise in FP64; few: the configuration for one
// or two CTAs per SM (two-step operand prefetch).
cudaError_t launch_syl_ws(int block, int nu, bool lyap, bool df, const Operands &o, const Sched &s, const Launch &l,
                          cudaStream_t st, bool few);

// Cholesky with warp-specialised CTAs (block B, nu update warps plus one
// diagonal warp); df: double-float update warps (SS_MODE_DF).
cudaError_t launch_potrf_ws(int block, int nu, bool df, const Operands &o, const Sched &s, const Launch &l,
                            cudaStream_t st, bool few);

// Solve stage of the SPD solve (R^T Y = B, R X = Y) over the valid instances
// of a binning pass, on queue head `group`; df: double-float block updates
// (SS_MODE_DF), the diagonal solves FP64.
cudaError_t launch_posv_solve(const int *d_n, const int *d_k, int max_k, const double *const *d_R, const int *d_ldr,
                              const double *const *d_B, const int *d_ldb, double *const *d_X, const int *d_ldx,
                              int *d_info, const Sched &s, int group, int batch, cudaStream_t st, bool df);

// Number of SMs of the current device (cached per device).
int sm_count();

}  // namespace ss
