// C ABI of the library (declared in include/smallsolve.h): argument checks,
// configuration selection, workspace layout and the launch plan of one call
// (binning pre-pass, then one persistent solve launch per launch group).
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "ss_internal.h"

namespace ss {

cudaError_t launch_potrf_fp64(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st);
cudaError_t launch_syl_fp64(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st, bool lyap);
cudaError_t launch_syl_ws(int block, int nu, bool lyap, bool df, const Operands &o, const Sched &s, const Launch &l,
                          cudaStream_t st, bool few);
cudaError_t launch_potrf_ws(int block, int nu, bool df, const Operands &o, const Sched &s, const Launch &l,
                            cudaStream_t st, bool few);
cudaError_t launch_mixed(int op, const Operands &o, const Sched &s, const Launch &l, cudaStream_t st);
int mixed_config_count(int op, int mode);
const Config *mixed_config_get(int op, int mode, int cfg);
long long mixed_scratch_per_n2(int op, int mode);
int mixed_launches(int op, int mode, int cfg);

namespace {

// FP64 configurations per operation: (block B, threads per CTA, variant).
// variant 0: CTA-wide diagonal-block work; 1: one warp does the diagonal
// blocks between CTA-wide updates (shorter dependent chain); 2: warp-
// specialised pipeline, one diagonal warp and (threads-32)/32 update warps;
// 3 (Cholesky): right-looking in shared memory for n <= block (64), the
// variant-1 blocked path above.  At most eight per operation (the learned
// selector predicts one time per configuration slot).
const Config kFp64Potrf[] = {
    {16, 96, 2}, {16, 64, 0}, {16, 160, 2}, {32, 128, 0}, {32, 256, 0},
    {16, 64, 1}, {16, 128, 1}, {64, 128, 3},
};
const Config kFp64Syl[] = {
    {8, 64, 0}, {16, 64, 0}, {16, 128, 0}, {32, 128, 0},
    {16, 128, 1}, {16, 160, 2}, {16, 96, 2}, {16, 64, 2},
};
constexpr int kNumFp64Potrf = sizeof(kFp64Potrf) / sizeof(kFp64Potrf[0]);
constexpr int kNumFp64Syl = sizeof(kFp64Syl) / sizeof(kFp64Syl[0]);
// SS_MODE_DF: variant 4, the warp-specialised pipeline with double-float
// update warps (Sylvester / Lyapunov: double-float diagonal blocks too;
// Cholesky: FP64 diagonal warp).
// Variant bit 3: for one or two CTAs per SM (few, large instances): all of
// the registers, and for Sylvester / Lyapunov the two-step operand prefetch.
const Config kDfSyl[] = {{16, 64, 4}, {16, 96, 4}, {16, 160, 4}, {16, 160, 12}, {16, 288, 12}, {32, 288, 12}};
const Config kDfPotrf[] = {{16, 96, 4}, {16, 160, 4}, {16, 160, 12}};
constexpr int kNumDfSyl = sizeof(kDfSyl) / sizeof(kDfSyl[0]);
constexpr int kNumDfPotrf = sizeof(kDfPotrf) / sizeof(kDfPotrf[0]);
// Mode ids 0..SS_MODE_DF index the per-mode tables (SS_MODE_AUTO's slot unused).
constexpr int kModeSlots = SS_MODE_DF + 1;

int host_bin(int n) { int k = 0; while ((1 << k) < n) ++k; return k; }

bool valid_op(int op) { return op == SS_OP_POTRF || op == SS_OP_TRSYL || op == SS_OP_TRLYAP; }
bool valid_mode(int m) { return (m >= 0 && m < SS_NUM_MODES) || m == SS_MODE_DF; }
bool valid_call_mode(int m) { return valid_mode(m) || m == SS_MODE_AUTO; }
bool refined_or_fp64(int m)
{
    return m == SS_MODE_FP64 || m == SS_MODE_FP32_REFINED || m == SS_MODE_TF32_REFINED ||
           m == SS_MODE_BF16_REFINED || m == SS_MODE_DF;
}

struct TableState {
    std::mutex mu;
    int table[3][kModeSlots][NUM_BINS];
    int auto_mode[3][NUM_BINS];
    int auto_cfg[3][NUM_BINS];
    TableState()
    {
        for (auto &a : table) for (auto &b : a) for (int &c : b) c = -1;
        for (auto &a : auto_mode) for (int &c : a) c = -1;
        for (auto &a : auto_cfg) for (int &c : a) c = -1;
    }
};
TableState &tables()
{
    static TableState t;
    return t;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

std::atomic<long long> g_launches{0};

// Auxiliary streams of one device: launch groups 2..k of a call run on them,
// forked from and joined back to the caller's stream with events, so that the
// persistent kernels of different groups overlap (one group's CTAs fill the
// SM slots another group's drained CTAs free).  Created once per device on
// first use; they hold no device memory.
constexpr int kAux = 3;
struct AuxPool {
    bool ready = false;
    cudaStream_t aux[kAux];
    cudaEvent_t fork;
    cudaEvent_t join[kAux];
};
std::mutex g_aux_mu;
AuxPool g_aux[64];

AuxPool *aux_pool()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    AuxPool &p = g_aux[dev];
    if (!p.ready) {
        for (int i = 0; i < kAux; ++i) {
            if (cudaStreamCreateWithFlags(&p.aux[i], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
            if (cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming) != cudaSuccess) return nullptr;
        }
        if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        p.ready = true;
    }
    return &p;
}

struct Profile {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;   // pairs: 2*i start, 2*i+1 stop
    int used = 0;                    // pairs recorded since the last read
};
Profile &profile()
{
    static Profile p;
    return p;
}

// Returns the event pair for this call, or false when profiling is off.
bool profile_pair(cudaEvent_t *a, cudaEvent_t *b)
{
    Profile &p = profile();
    std::lock_guard<std::mutex> g(p.mu);
    if (!p.on) return false;
    if ((int)p.pool.size() < 2 * (p.used + 1)) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return false;
        if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return false; }
        p.pool.push_back(e0);
        p.pool.push_back(e1);
    }
    *a = p.pool[2 * p.used];
    *b = p.pool[2 * p.used + 1];
    ++p.used;
    return true;
}

}  // namespace

int config_count(int op, int mode)
{
    if (mode == SS_MODE_FP64) return op == SS_OP_POTRF ? kNumFp64Potrf : kNumFp64Syl;
    if (mode == SS_MODE_DF) return op == SS_OP_POTRF ? kNumDfPotrf : kNumDfSyl;
    return mixed_config_count(op, mode);
}

const Config *config_get(int op, int mode, int cfg)
{
    if (cfg < 0 || cfg >= config_count(op, mode)) return nullptr;
    if (mode == SS_MODE_FP64) return op == SS_OP_POTRF ? &kFp64Potrf[cfg] : &kFp64Syl[cfg];
    if (mode == SS_MODE_DF) return op == SS_OP_POTRF ? &kDfPotrf[cfg] : &kDfSyl[cfg];
    return mixed_config_get(op, mode, cfg);
}

// Built-in default: a single configuration chosen from the largest order.
// Built-in FP64 defaults, from the autotuner's timings on GB300 (fastest
// configuration per size bin, batches 64..2048):
//   Cholesky: one-warp diagonal blocks (B = 16) up to n = 16, then the
//   warp-specialised pipeline with two update warps (large batches up to
//   n = 128) or four;
//   Sylvester / Lyapunov: CTA-wide B = 8 / 16 up to n = 32, warp-specialised
//   with one update warp up to 64, then two (large batches) or four.
int config_default(int op, int mode, int max_n, int batch)
{
    if (mode == SS_MODE_DF) return op == SS_OP_POTRF ? 0 : 2;   // (16, 96, 4) / (16, 160, 4)
    if (mode != SS_MODE_FP64) return 0;
    if (op == SS_OP_POTRF) {
        if (max_n <= 16) return 5;                       // (16, 64, 1)
        if (max_n <= 128 && batch >= 1024) return 0;     // (16, 96, 2)
        return 2;                                        // (16, 160, 2)
    }
    if (max_n <= 8) return 0;             // (8, 64, 0)
    if (max_n <= 32) return 1;            // (16, 64, 0)
    if (max_n <= 64) return 7;            // (16, 64, 2)
    if (max_n <= 128 && batch >= 1024) return 6;   // (16, 96, 2)
    return 5;                             // (16, 160, 2)
}

int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (cache[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = v > 0 ? v : 1;
    }
    return cache[dev];
}

// SS_MODE_DF scratch: Sylvester / Lyapunov the pre-split double-float copies
// of L, U and X (3 pairs per n^2, the bound of m^2 + n^2 + m n for
// max(m, n) = n); Cholesky X as pairs (1 pair per n^2).
static long long df_scratch_per_n2(int op) { return op != SS_OP_POTRF ? 6 : 2; }

static long long scratch_per_n2(int op, int mode)
{
    if (mode == SS_MODE_AUTO) {
        long long m = df_scratch_per_n2(op);
        for (int md = 1; md < SS_NUM_MODES; ++md) {
            const long long v = mixed_scratch_per_n2(op, md);
            if (v > m) m = v;
        }
        return m;
    }
    if (mode == SS_MODE_DF) return df_scratch_per_n2(op);
    return mode == SS_MODE_FP64 ? 0 : mixed_scratch_per_n2(op, mode);
}

static bool has_df(int mode) { return mode == SS_MODE_DF || mode == SS_MODE_AUTO; }

// Workspace layout: [meta: META_INTS ints][perm: batch ints][dfs: batch
// DfInst, SS_MODE_DF and AUTO][scr: batch int64][scratch: batch * max_n^2 *
// scratch_per_n2 floats], each part aligned to 256 bytes.
size_t workspace_bytes(int op, int batch, int max_n, int mode)
{
    size_t b = align_up(META_INTS * sizeof(int), 256);
    b += align_up((size_t)batch * sizeof(int), 256);
    if (has_df(mode)) b += align_up((size_t)batch * sizeof(DfInst), 256);
    const long long per = scratch_per_n2(op, mode);
    if (per > 0) {
        b += align_up((size_t)batch * sizeof(long long), 256);
        b += align_up((size_t)batch * (size_t)max_n * (size_t)max_n * (size_t)per * sizeof(float), 256);
    }
    return b;
}

void carve_workspace(void *d_work, size_t work_bytes, int op, int batch, int max_n, int mode, Sched *s)
{
    (void)max_n;
    char *p = static_cast<char *>(d_work);
    s->meta = reinterpret_cast<int *>(p);
    p += align_up(META_INTS * sizeof(int), 256);
    s->perm = reinterpret_cast<const int *>(p);
    p += align_up((size_t)batch * sizeof(int), 256);
    s->dfs = nullptr;
    if (has_df(mode)) {
        s->dfs = reinterpret_cast<const DfInst *>(p);
        p += align_up((size_t)batch * sizeof(DfInst), 256);
    }
    s->scr = nullptr;
    s->scratch = nullptr;
    s->scratch_elems = 0;
    if (scratch_per_n2(op, mode) > 0) {
        s->scr = reinterpret_cast<const long long *>(p);
        p += align_up((size_t)batch * sizeof(long long), 256);
        s->scratch = p;
        s->scratch_elems = (long long)(((static_cast<char *>(d_work) + work_bytes) - p) / sizeof(float));
    }
}

}  // namespace ss

using namespace ss;

namespace {

// Shared driver of the three entry points.
// max_n: the host bound of d_n; for the rectangular Sylvester solve (o.m set)
// also max_m, and sizes are keyed by max(m, n).
int run(int op, int batch, int max_n, const Operands &o, int mode, int cfg, void *d_work,
        size_t work_bytes, void *stream, int arg_mode, int arg_work, int max_m = 0)
{
    const int max_key = (o.m != nullptr && max_m > max_n) ? max_m : max_n;
    if (!valid_call_mode(mode)) return -arg_mode;
    const bool autom = mode == SS_MODE_AUTO;
    const int ncfg = autom ? 1 : config_count(op, mode);
    if (ncfg <= 0) return -arg_mode;
    if (!autom && !(cfg == SS_CFG_DEFAULT || cfg == SS_CFG_TABLE || (cfg >= 0 && cfg < ncfg)))
        return -(arg_mode + 1);
    if (batch == 0) return 0;
    const size_t need = workspace_bytes(op, batch, max_key, mode);
    if (d_work == nullptr) return -arg_work;
    if (work_bytes < need) return -(arg_work + 1);

    // (mode, configuration) per size bin, then launch groups = runs of equal pairs.
    int mode_of_bin[NUM_BINS], by_bin[NUM_BINS];
    const int top = host_bin(max_key > 0 ? max_key : 1);
    for (int k = 0; k < NUM_BINS; ++k) {
        int md = mode, c = -1;
        if (autom) {
            std::lock_guard<std::mutex> g(tables().mu);
            md = tables().auto_mode[op][k];
            c = tables().auto_cfg[op][k];
            if (md < 0 || !refined_or_fp64(md) || config_count(op, md) <= 0) { md = SS_MODE_FP64; c = -1; }
        } else if (cfg >= 0) {
            c = cfg;
        } else if (cfg == SS_CFG_TABLE) {
            std::lock_guard<std::mutex> g(tables().mu);
            c = tables().table[op][mode][k];
        }
        if (c < 0 || c >= config_count(op, md)) c = config_default(op, md, max_key, batch);
        mode_of_bin[k] = md;
        by_bin[k] = c;
    }
    int group_of_bin[NUM_BINS];
    int group_cfg[MAX_GROUPS], group_mode[MAX_GROUPS];
    int ngroups = 0;
    for (int k = NUM_BINS - 1; k >= 0; --k) {
        if (k > top) { group_of_bin[k] = -1; continue; }
        if (ngroups > 0 && group_cfg[ngroups - 1] == by_bin[k] && group_mode[ngroups - 1] == mode_of_bin[k]) {
            group_of_bin[k] = ngroups - 1;
        } else {
            if (ngroups == MAX_GROUPS) return SS_ERR_CUDA;
            group_cfg[ngroups] = by_bin[k];
            group_mode[ngroups] = mode_of_bin[k];
            group_of_bin[k] = ngroups++;
        }
    }

    Sched s;
    carve_workspace(d_work, work_bytes, op, batch, max_key, mode, &s);
    const long long per = scratch_per_n2(op, mode);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_binning(batch, max_n, o.n, o.info, s, group_of_bin, ngroups, per, st, o.m, max_m);
    if (e != cudaSuccess) return SS_ERR_CUDA;
    // A double-float group is the zero-shift pipeline and the rescaled pass;
    // for Sylvester / Lyapunov also the range fix-up pass.
    int nlaunch = 1 + ngroups;
    for (int g = 0; g < ngroups; ++g) {
        if (group_mode[g] == SS_MODE_DF) {
            if (s.dfs == nullptr) return SS_ERR_CUDA;
            nlaunch += op != SS_OP_POTRF ? 2 : 1;
        } else if (group_mode[g] != SS_MODE_FP64) {
            nlaunch += mixed_launches(op, group_mode[g], group_cfg[g]) - 1;
        }
    }
    g_launches.fetch_add(nlaunch, std::memory_order_relaxed);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const bool prof = profile_pair(&ev0, &ev1);
    if (prof) cudaEventRecord(ev0, st);
    // Groups beyond the first go to auxiliary streams forked after the pre-pass.
    std::unique_lock<std::mutex> aux_lock(g_aux_mu, std::defer_lock);
    AuxPool *ap = nullptr;
    if (ngroups > 1) {
        aux_lock.lock();
        ap = aux_pool();
        if (ap && cudaEventRecord(ap->fork, st) != cudaSuccess) ap = nullptr;
        if (ap)
            for (int i = 0; i < kAux && i < ngroups - 1; ++i)
                if (cudaStreamWaitEvent(ap->aux[i], ap->fork, 0) != cudaSuccess) { ap = nullptr; break; }
    }
    for (int g = 0; g < ngroups; ++g) {
        Launch l{g, group_cfg[g], group_mode[g], max_key, batch};
        cudaStream_t gs = (g == 0 || ap == nullptr) ? st : ap->aux[(g - 1) % kAux];
        if (l.mode == SS_MODE_FP64) {
            if (op == SS_OP_POTRF) e = launch_potrf_fp64(o, s, l, gs);
            else e = launch_syl_fp64(o, s, l, gs, op == SS_OP_TRLYAP);
        } else if (l.mode == SS_MODE_DF) {
            const Config *c = config_get(op, SS_MODE_DF, l.cfg);
            if (!c) e = cudaErrorInvalidValue;
            else if (op == SS_OP_POTRF) e = launch_potrf_ws(c->block, (c->threads - 32) / 32, true, o, s, l, gs,
                                                            (c->variant & 8) != 0);
            else e = launch_syl_ws(c->block, (c->threads - 32) / 32, op == SS_OP_TRLYAP, true, o, s, l, gs,
                                   (c->variant & 8) != 0);
        } else {
            e = launch_mixed(op, o, s, l, gs);
        }
        if (e != cudaSuccess) return SS_ERR_CUDA;
    }
    if (ap) {
        for (int i = 0; i < kAux && i < ngroups - 1; ++i) {
            if (cudaEventRecord(ap->join[i], ap->aux[i]) != cudaSuccess) return SS_ERR_CUDA;
            if (cudaStreamWaitEvent(st, ap->join[i], 0) != cudaSuccess) return SS_ERR_CUDA;
        }
    }
    if (prof) cudaEventRecord(ev1, st);
    return 0;
}

}  // namespace

extern "C" {

int potrf_upper(int batch, int max_n, const int *d_n, const double *const *d_A, const int *d_lda,
                double *const *d_X, const int *d_ldx, int *d_info, int mode, int cfg,
                void *d_work, size_t work_bytes, void *stream)
{
    if (batch < 0) return -1;
    if (max_n < 0 || max_n > SS_MAX_N) return -2;
    if (batch > 0) {
        if (!d_n) return -3;
        if (!d_A) return -4;
        if (!d_lda) return -5;
        if (!d_X) return -6;
        if (!d_ldx) return -7;
        if (!d_info) return -8;
    }
    Operands o{d_n, d_A, d_lda, nullptr, nullptr, nullptr, nullptr, d_X, d_ldx, d_info};
    return run(SS_OP_POTRF, batch, max_n, o, mode, cfg, d_work, work_bytes, stream, 9, 11);
}

int trsyl_lu(int batch, int max_n, const int *d_n, const double *const *d_L, const int *d_ldl,
             const double *const *d_U, const int *d_ldu, const double *const *d_C, const int *d_ldc,
             double *const *d_X, const int *d_ldx, int *d_info, int mode, int cfg, void *d_work,
             size_t work_bytes, void *stream)
{
    if (batch < 0) return -1;
    if (max_n < 0 || max_n > SS_MAX_N) return -2;
    if (batch > 0) {
        if (!d_n) return -3;
        if (!d_L) return -4;
        if (!d_ldl) return -5;
        if (!d_U) return -6;
        if (!d_ldu) return -7;
        if (!d_C) return -8;
        if (!d_ldc) return -9;
        if (!d_X) return -10;
        if (!d_ldx) return -11;
        if (!d_info) return -12;
    }
    Operands o{d_n, d_L, d_ldl, d_U, d_ldu, d_C, d_ldc, d_X, d_ldx, d_info};
    return run(SS_OP_TRSYL, batch, max_n, o, mode, cfg, d_work, work_bytes, stream, 13, 15);
}

int trsyl_rect(int batch, int max_m, int max_n, const int *d_m, const int *d_n, const double *const *d_L,
               const int *d_ldl, const double *const *d_U, const int *d_ldu, const double *const *d_C,
               const int *d_ldc, double *const *d_X, const int *d_ldx, int *d_info, int mode, int cfg,
               void *d_work, size_t work_bytes, void *stream)
{
    if (batch < 0) return -1;
    if (max_m < 0 || max_m > SS_MAX_N) return -2;
    if (max_n < 0 || max_n > SS_MAX_N) return -3;
    if (batch > 0) {
        if (!d_m) return -4;
        if (!d_n) return -5;
        if (!d_L) return -6;
        if (!d_ldl) return -7;
        if (!d_U) return -8;
        if (!d_ldu) return -9;
        if (!d_C) return -10;
        if (!d_ldc) return -11;
        if (!d_X) return -12;
        if (!d_ldx) return -13;
        if (!d_info) return -14;
    }
    if (mode != SS_MODE_FP64 && mode != SS_MODE_DF) return -15;
    Operands o{d_n, d_L, d_ldl, d_U, d_ldu, d_C, d_ldc, d_X, d_ldx, d_info, d_m};
    return run(SS_OP_TRSYL, batch, max_n, o, mode, cfg, d_work, work_bytes, stream, 15, 17, max_m);
}

int posv_upper(int batch, int max_n, int max_k, const int *d_n, const int *d_k, const double *const *d_A,
               const int *d_lda, double *const *d_R, const int *d_ldr, const double *const *d_B,
               const int *d_ldb, double *const *d_X, const int *d_ldx, int *d_info, int mode, int cfg,
               void *d_work, size_t work_bytes, void *stream)
{
    if (batch < 0) return -1;
    if (max_n < 0 || max_n > SS_MAX_N) return -2;
    if (max_k < 0) return -3;
    if (batch > 0) {
        if (!d_n) return -4;
        if (!d_k) return -5;
        if (!d_A) return -6;
        if (!d_lda) return -7;
        if (!d_R) return -8;
        if (!d_ldr) return -9;
        if (!d_B) return -10;
        if (!d_ldb) return -11;
        if (!d_X) return -12;
        if (!d_ldx) return -13;
        if (!d_info) return -14;
    }
    if (mode != SS_MODE_FP64 && mode != SS_MODE_DF) return -15;
    // Stage 1: the factor R (R^T R = A) by the Cholesky path (FP64 or DF); it also
    // sorts the instances by n and leaves the order in the workspace.
    Operands o{d_n, d_A, d_lda, nullptr, nullptr, nullptr, nullptr, d_R, d_ldr, d_info};
    const int rc = run(SS_OP_POTRF, batch, max_n, o, mode, cfg, d_work, work_bytes, stream, 15, 17);
    if (rc != 0 || batch == 0) return rc;
    // Stage 2: the two triangular solves, on the last queue head (the factor
    // uses at most NUM_BINS < MAX_GROUPS launch groups).
    Sched s;
    carve_workspace(d_work, work_bytes, SS_OP_POTRF, batch, max_n, mode, &s);
    cudaError_t e = launch_posv_solve(d_n, d_k, max_k, d_R, d_ldr, d_B, d_ldb, d_X, d_ldx, d_info, s,
                                      MAX_GROUPS - 1, batch, static_cast<cudaStream_t>(stream), mode == SS_MODE_DF);
    if (e != cudaSuccess) return SS_ERR_CUDA;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return 0;
}

int trlyap_l(int batch, int max_n, const int *d_n, const double *const *d_L, const int *d_ldl,
             const double *const *d_S, const int *d_lds, double *const *d_X, const int *d_ldx,
             int *d_info, int mode, int cfg, void *d_work, size_t work_bytes, void *stream)
{
    if (batch < 0) return -1;
    if (max_n < 0 || max_n > SS_MAX_N) return -2;
    if (batch > 0) {
        if (!d_n) return -3;
        if (!d_L) return -4;
        if (!d_ldl) return -5;
        if (!d_S) return -6;
        if (!d_lds) return -7;
        if (!d_X) return -8;
        if (!d_ldx) return -9;
        if (!d_info) return -10;
    }
    Operands o{d_n, d_L, d_ldl, nullptr, nullptr, d_S, d_lds, d_X, d_ldx, d_info};
    return run(SS_OP_TRLYAP, batch, max_n, o, mode, cfg, d_work, work_bytes, stream, 11, 13);
}

int ss_workspace_size(int op, int batch, int max_n, int mode, size_t *bytes)
{
    if (!valid_op(op)) return -1;
    if (batch < 0) return -2;
    if (max_n < 0 || max_n > SS_MAX_N) return -3;
    if (!valid_call_mode(mode)) return -4;
    if (!bytes) return -5;
    *bytes = workspace_bytes(op, batch, max_n, mode);
    return 0;
}

int ss_config_count(int op, int mode)
{
    if (!valid_op(op)) return -1;
    if (!valid_mode(mode)) return -2;
    return config_count(op, mode);
}

int ss_config_describe(int op, int mode, int cfg, int *block, int *threads, int *variant)
{
    if (!valid_op(op)) return -1;
    if (!valid_mode(mode)) return -2;
    const Config *c = config_get(op, mode, cfg);
    if (!c) return -3;
    if (block) *block = c->block;
    if (threads) *threads = c->threads;
    if (variant) *variant = c->variant;
    return 0;
}

int ss_set_config_table(int op, int mode, int nbins, const int *cfg_by_bin)
{
    if (!valid_op(op)) return -1;
    if (!valid_mode(mode)) return -2;
    if (nbins < 0 || nbins > NUM_BINS) return -3;
    if (nbins > 0 && !cfg_by_bin) return -4;
    const int ncfg = config_count(op, mode);
    for (int k = 0; k < nbins; ++k)
        if (cfg_by_bin[k] < -1 || cfg_by_bin[k] >= ncfg) return -4;
    std::lock_guard<std::mutex> g(tables().mu);
    for (int k = 0; k < NUM_BINS; ++k) tables().table[op][mode][k] = k < nbins ? cfg_by_bin[k] : -1;
    return 0;
}

int ss_set_auto_table(int op, int nbins, const int *mode_by_bin, const int *cfg_by_bin)
{
    if (!valid_op(op)) return -1;
    if (nbins < 0 || nbins > NUM_BINS) return -2;
    if (nbins > 0 && !mode_by_bin) return -3;
    if (nbins > 0 && !cfg_by_bin) return -4;
    for (int k = 0; k < nbins; ++k) {
        const int md = mode_by_bin[k];
        if (md == -1) continue;
        if (!refined_or_fp64(md) || config_count(op, md) <= 0) return -3;
        if (cfg_by_bin[k] < -1 || cfg_by_bin[k] >= config_count(op, md)) return -4;
    }
    std::lock_guard<std::mutex> g(tables().mu);
    for (int k = 0; k < NUM_BINS; ++k) {
        tables().auto_mode[op][k] = k < nbins ? mode_by_bin[k] : -1;
        tables().auto_cfg[op][k] = k < nbins ? cfg_by_bin[k] : -1;
    }
    return 0;
}

int ss_version(void) { return 1; }

long long ss_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int ss_profile_enable(int on)
{
    Profile &p = profile();
    std::lock_guard<std::mutex> g(p.mu);
    p.on = on != 0;
    return 0;
}

int ss_profile_read(double *total_ms, int *calls)
{
    if (!total_ms) return -1;
    if (!calls) return -2;
    Profile &p = profile();
    std::lock_guard<std::mutex> g(p.mu);
    double t = 0.0;
    for (int i = 0; i < p.used; ++i) {
        if (cudaEventSynchronize(p.pool[2 * i + 1]) != cudaSuccess) return SS_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.pool[2 * i], p.pool[2 * i + 1]) != cudaSuccess) return SS_ERR_CUDA;
        t += ms;
    }
    *total_ms = t;
    *calls = p.used;
    p.used = 0;
    return 0;
}

}  // extern "C"
