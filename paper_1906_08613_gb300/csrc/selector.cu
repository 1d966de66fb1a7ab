// The learned selector and the autotuner behind the C ABI (declared in
// include/smallsolve.h).
//
// The paper's generator finds the fastest code by an autotuning loop over
// algorithm variants and implementation parameters ("Generator structure"
// paragraph), and names a model-based replacement for that loop as future
// work ("Limitations and future work" paragraph).  ss_autotune is the loop:
// it times every configuration of one precision mode on the caller's batch.
// The selector is the model: an MLP cost model (the network of mlp.cu) that
// predicts the log2 run time of every configuration of every precision mode
// for a bucket of (operation, order n, number of instances), trained on the
// autotuner's timings by the library's own forward / backward / Adam
// kernels; its argmin picks the (mode, cfg) of each size bin, which
// ss_selector_install writes into the SS_MODE_AUTO table.
//
// The decision from a set of predictions is plain host code
// (ss_selector_queries -> network -> ss_selector_decide), so it can be
// checked without a GPU; ss_selector_predict runs the network on the GPU in
// between.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "ss_internal.h"

namespace ss {
namespace {

// The selector's precision modes, in feature order.
constexpr int kSelModes = 5;
const int kModeIds[kSelModes] = {SS_MODE_FP64, SS_MODE_FP32_REFINED, SS_MODE_TF32_REFINED, SS_MODE_BF16_REFINED,
                                 SS_MODE_DF};
constexpr int kOps = 3;
constexpr int kMaxRows = SS_NUM_BINS * kSelModes;

struct Model {
    bool ready = false;
    std::vector<float> params = std::vector<float>(SS_MLP_PARAMS, 0.0f);
    // Configurations of (op, mode) that had training targets; a slot that
    // never had one carries no information, so choices stay below it.
    int cfg_count[kOps][kSelModes] = {};
    // Largest batch the network was trained on per (op, size bin, mode); 0:
    // none recorded (no limit).  Beyond it a prediction is taken at that
    // batch and scaled by count / batch (the kernels are throughput-bound
    // there, a regime the network, trained on smaller batches, does not
    // extrapolate to).
    int batch_max[kOps][SS_NUM_BINS][kSelModes] = {};
    unsigned long long version = 0;
};

std::mutex g_mu;
Model g_model;
unsigned long long g_next_version = 1;

// Per-device copies of the parameters and the row buffers of one prediction
// (allocated on a device's first prediction, kept until exit).
struct DevState {
    float *p = nullptr, *x = nullptr, *y = nullptr;
    unsigned long long version = 0;
};
DevState g_dev[64];

int host_bin(int n) { int k = 0; while ((1 << k) < n) ++k; return k; }

double bin_center(int k)
{
    if (k == 0) return 1.0;
    const double lo = (double)((1 << (k - 1)) + 1), hi = (double)(1 << k);
    return sqrt(lo * hi);
}

// Feature row: op one-hot, log2(n) / 9, log2(batch) / 14, mode one-hot.
void features(int op, double n, double batch, int mi, float *f)
{
    for (int i = 0; i < SS_MLP_IN; ++i) f[i] = 0.0f;
    f[op] = 1.0f;
    f[3] = (float)(log2(n > 1.0 ? n : 1.0) / 9.0);
    f[4] = (float)(log2(batch > 1.0 ? batch : 1.0) / 14.0);
    f[5 + mi] = 1.0f;
}

int n_cfgs(const Model &m, int op, int mi)
{
    const int cnt = config_count(op, kModeIds[mi]);
    return std::min(cnt, m.cfg_count[op][mi]);
}

// (batch fed to the network, factor on its prediction) for `count`
// instances in size bin k.
void query_batch(const Model &m, int op, int k, double count, int mi, double *fb, double *scale)
{
    const int bmax = m.batch_max[op][k][mi];
    if (bmax > 0 && count > bmax) {
        *fb = bmax;
        *scale = count / bmax;
    } else {
        *fb = count;
        *scale = 1.0;
    }
}

struct Row {
    int k, mi, cnt;
    double scale;
};

// The rows to evaluate for a call with count_by_bin[k] instances in bin k:
// every (bin with instances, mode with configurations) pair, bins ascending,
// modes in feature order.
std::vector<Row> make_rows(const Model &m, int op, int nbins, const int *counts, float *x)
{
    std::vector<Row> rows;
    for (int k = 0; k < nbins; ++k) {
        if (counts[k] <= 0) continue;
        for (int mi = 0; mi < kSelModes; ++mi) {
            const int cnt = n_cfgs(m, op, mi);
            if (cnt <= 0) continue;
            double fb, scale;
            query_batch(m, op, k, counts[k], mi, &fb, &scale);
            if (x) features(op, bin_center(k), fb, mi, x + rows.size() * SS_MLP_IN);
            rows.push_back(Row{k, mi, cnt, scale});
        }
    }
    return rows;
}

// Choice from the predictions y[row * SS_MLP_OUT + cfg] (log2 ms).
//   SS_SELECTOR_PER_BIN: per bin, the (mode, cfg) of the smallest predicted
//     time (first mode wins ties);
//   SS_SELECTOR_CALL: one (mode, cfg) for the whole call, the smallest
//     predicted total over the call's bins, written to every bin.  One
//     launch keeps all sizes in one persistent queue whose longest-first
//     order balances the SMs; a choice per bin splits the call into launch
//     groups, each with its own tail.
int decide(const Model &m, int op, int nbins, const int *counts, int policy, const float *y, int *modes, int *cfgs,
           double *pred_ms)
{
    const std::vector<Row> rows = make_rows(m, op, nbins, counts, nullptr);
    for (int k = 0; k < nbins; ++k) {
        modes[k] = -1;
        cfgs[k] = -1;
    }
    double total = 0.0;
    if (policy == SS_SELECTOR_PER_BIN) {
        std::vector<double> best(nbins, INFINITY);
        for (size_t r = 0; r < rows.size(); ++r) {
            const float *yr = y + r * SS_MLP_OUT;
            int c = 0;
            for (int j = 1; j < rows[r].cnt; ++j)
                if (yr[j] < yr[c]) c = j;
            const double v = (double)yr[c] + log2(rows[r].scale);
            const int k = rows[r].k;
            if (v < best[k]) {
                best[k] = v;
                modes[k] = kModeIds[rows[r].mi];
                cfgs[k] = c;
            }
        }
        for (int k = 0; k < nbins; ++k)
            if (modes[k] >= 0) total += exp2(best[k]);
    } else {
        double best = INFINITY;
        int bm = -1, bc = -1;
        for (int mi = 0; mi < kSelModes; ++mi) {
            double tot[SS_MLP_OUT] = {0};
            int cnt = 0;
            bool any = false;
            for (size_t r = 0; r < rows.size(); ++r) {
                if (rows[r].mi != mi) continue;
                any = true;
                cnt = rows[r].cnt;
                for (int j = 0; j < cnt; ++j) tot[j] += rows[r].scale * exp2((double)y[r * SS_MLP_OUT + j]);
            }
            if (!any) continue;
            int c = 0;
            for (int j = 1; j < cnt; ++j)
                if (tot[j] < tot[c]) c = j;
            if (tot[c] < best) {
                best = tot[c];
                bm = kModeIds[mi];
                bc = c;
            }
        }
        if (bm >= 0)
            for (int k = 0; k < nbins; ++k) {
                modes[k] = bm;
                cfgs[k] = bc;
            }
        total = bm >= 0 ? best : 0.0;
    }
    if (pred_ms) *pred_ms = total;
    return 0;
}

// The GPU copies of the current model for the current device.
DevState *device_state(const Model &m)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    DevState &d = g_dev[dev];
    if (!d.p) {
        if (cudaMalloc(&d.p, SS_MLP_PARAMS * sizeof(float)) != cudaSuccess) return nullptr;
        if (cudaMalloc(&d.x, kMaxRows * SS_MLP_IN * sizeof(float)) != cudaSuccess) return nullptr;
        if (cudaMalloc(&d.y, kMaxRows * SS_MLP_OUT * sizeof(float)) != cudaSuccess) return nullptr;
    }
    if (d.version != m.version) {
        if (cudaMemcpy(d.p, m.params.data(), SS_MLP_PARAMS * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return nullptr;
        d.version = m.version;
    }
    return &d;
}

const char kMagic[8] = {'S', 'S', 'M', 'L', 'P', '1', 0, 0};

}  // namespace
}  // namespace ss

using namespace ss;

extern "C" {

int ss_selector_set(const float *h_params, const int *cfg_count, const int *batch_max)
{
    if (!h_params) return -1;
    for (int i = 0; i < SS_MLP_PARAMS; ++i)
        if (!isfinite(h_params[i])) return -1;
    if (cfg_count)
        for (int i = 0; i < kOps * kSelModes; ++i)
            if (cfg_count[i] < 0 || cfg_count[i] > SS_MLP_OUT) return -2;
    if (batch_max)
        for (int i = 0; i < kOps * SS_NUM_BINS * kSelModes; ++i)
            if (batch_max[i] < 0) return -3;
    std::lock_guard<std::mutex> g(g_mu);
    Model &m = g_model;
    m.params.assign(h_params, h_params + SS_MLP_PARAMS);
    for (int op = 0; op < kOps; ++op)
        for (int mi = 0; mi < kSelModes; ++mi) {
            m.cfg_count[op][mi] = cfg_count ? cfg_count[op * kSelModes + mi]
                                            : std::min(config_count(op, kModeIds[mi]), SS_MLP_OUT);
            for (int k = 0; k < SS_NUM_BINS; ++k)
                m.batch_max[op][k][mi] = batch_max ? batch_max[(op * SS_NUM_BINS + k) * kSelModes + mi] : 0;
        }
    m.ready = true;
    m.version = g_next_version++;
    return 0;
}

int ss_selector_get(float *h_params, int *cfg_count, int *batch_max)
{
    std::lock_guard<std::mutex> g(g_mu);
    const Model &m = g_model;
    if (!m.ready) return -1;
    if (h_params) memcpy(h_params, m.params.data(), SS_MLP_PARAMS * sizeof(float));
    for (int op = 0; op < kOps; ++op)
        for (int mi = 0; mi < kSelModes; ++mi) {
            if (cfg_count) cfg_count[op * kSelModes + mi] = m.cfg_count[op][mi];
            if (batch_max)
                for (int k = 0; k < SS_NUM_BINS; ++k) batch_max[(op * SS_NUM_BINS + k) * kSelModes + mi] = m.batch_max[op][k][mi];
        }
    return 0;
}

int ss_selector_clear(void)
{
    std::lock_guard<std::mutex> g(g_mu);
    g_model.ready = false;
    return 0;
}

int ss_selector_save(const char *path)
{
    if (!path) return -1;
    std::lock_guard<std::mutex> g(g_mu);
    const Model &m = g_model;
    if (!m.ready) return -1;
    FILE *f = fopen(path, "wb");
    if (!f) return -1;
    const int dims[4] = {SS_MLP_IN, SS_MLP_HIDDEN, SS_MLP_OUT, SS_NUM_BINS};
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(dims, sizeof(int), 4, f) == 4 &&
              fwrite(m.params.data(), sizeof(float), SS_MLP_PARAMS, f) == (size_t)SS_MLP_PARAMS &&
              fwrite(m.cfg_count, sizeof(int), kOps * kSelModes, f) == (size_t)(kOps * kSelModes) &&
              fwrite(m.batch_max, sizeof(int), kOps * SS_NUM_BINS * kSelModes, f) ==
                  (size_t)(kOps * SS_NUM_BINS * kSelModes);
    ok = (fclose(f) == 0) && ok;
    return ok ? 0 : SS_ERR_IO;
}

int ss_selector_load(const char *path)
{
    if (!path) return -1;
    FILE *f = fopen(path, "rb");
    if (!f) return SS_ERR_IO;
    char magic[8];
    int dims[4];
    std::vector<float> p(SS_MLP_PARAMS);
    int cc[kOps * kSelModes], bm[kOps * SS_NUM_BINS * kSelModes];
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(dims, sizeof(int), 4, f) == 4 &&
              dims[0] == SS_MLP_IN && dims[1] == SS_MLP_HIDDEN && dims[2] == SS_MLP_OUT && dims[3] == SS_NUM_BINS &&
              fread(p.data(), sizeof(float), SS_MLP_PARAMS, f) == (size_t)SS_MLP_PARAMS &&
              fread(cc, sizeof(int), kOps * kSelModes, f) == (size_t)(kOps * kSelModes) &&
              fread(bm, sizeof(int), kOps * SS_NUM_BINS * kSelModes, f) == (size_t)(kOps * SS_NUM_BINS * kSelModes);
    fclose(f);
    if (!ok) return SS_ERR_IO;
    const int rc = ss_selector_set(p.data(), cc, bm);
    return rc == 0 ? 0 : SS_ERR_IO;
}

int ss_selector_queries(int op, int nbins, const int *count_by_bin, float *h_x, int *nrows)
{
    if (op < 0 || op >= kOps) return -1;
    if (nbins < 0 || nbins > SS_NUM_BINS) return -2;
    if (nbins > 0 && !count_by_bin) return -3;
    if (!nrows) return -5;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_model.ready) return SS_ERR_NO_SELECTOR;
    float x[kMaxRows * SS_MLP_IN];
    const std::vector<Row> rows = make_rows(g_model, op, nbins, count_by_bin, x);
    if (h_x) memcpy(h_x, x, rows.size() * SS_MLP_IN * sizeof(float));
    *nrows = (int)rows.size();
    return 0;
}

int ss_selector_decide(int op, int nbins, const int *count_by_bin, int policy, const float *h_y, int *mode_by_bin,
                       int *cfg_by_bin, double *pred_ms)
{
    if (op < 0 || op >= kOps) return -1;
    if (nbins < 0 || nbins > SS_NUM_BINS) return -2;
    if (nbins > 0 && !count_by_bin) return -3;
    if (policy != SS_SELECTOR_PER_BIN && policy != SS_SELECTOR_CALL) return -4;
    if (!h_y) return -5;
    if (nbins > 0 && !mode_by_bin) return -6;
    if (nbins > 0 && !cfg_by_bin) return -7;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_model.ready) return SS_ERR_NO_SELECTOR;
    return decide(g_model, op, nbins, count_by_bin, policy, h_y, mode_by_bin, cfg_by_bin, pred_ms);
}

int ss_selector_predict(int op, int nbins, const int *count_by_bin, int policy, int *mode_by_bin, int *cfg_by_bin,
                        double *pred_ms, void *stream)
{
    if (op < 0 || op >= kOps) return -1;
    if (nbins < 0 || nbins > SS_NUM_BINS) return -2;
    if (nbins > 0 && !count_by_bin) return -3;
    if (policy != SS_SELECTOR_PER_BIN && policy != SS_SELECTOR_CALL) return -4;
    if (nbins > 0 && !mode_by_bin) return -5;
    if (nbins > 0 && !cfg_by_bin) return -6;
    std::lock_guard<std::mutex> g(g_mu);
    const Model &m = g_model;
    if (!m.ready) return SS_ERR_NO_SELECTOR;
    float x[kMaxRows * SS_MLP_IN], y[kMaxRows * SS_MLP_OUT];
    const std::vector<Row> rows = make_rows(m, op, nbins, count_by_bin, x);
    const int nr = (int)rows.size();
    if (nr > 0) {
        DevState *d = device_state(m);
        if (!d) return SS_ERR_CUDA;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (cudaMemcpyAsync(d->x, x, (size_t)nr * SS_MLP_IN * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return SS_ERR_CUDA;
        if (ss_mlp_forward(d->p, nr, d->x, d->y, stream) != 0) return SS_ERR_CUDA;
        if (cudaMemcpyAsync(y, d->y, (size_t)nr * SS_MLP_OUT * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SS_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return SS_ERR_CUDA;
    }
    return decide(m, op, nbins, count_by_bin, policy, y, mode_by_bin, cfg_by_bin, pred_ms);
}

int ss_selector_install(int op, int nbins, const int *count_by_bin, int policy, void *stream)
{
    int modes[SS_NUM_BINS], cfgs[SS_NUM_BINS];
    const int rc = ss_selector_predict(op, nbins, count_by_bin, policy, modes, cfgs, nullptr, stream);
    if (rc != 0) return rc;
    return ss_set_auto_table(op, nbins, modes, cfgs);
}

int ss_selector_train(const float *h_x, const float *h_t, const float *h_m, int rows, const float *h_init, int steps,
                      float lr, float *h_loss, void *stream)
{
    if (!h_x) return -1;
    if (!h_t) return -2;
    if (!h_m) return -3;
    if (rows < 1) return -4;
    if (steps < 1) return -6;
    if (!(lr > 0.0f)) return -7;
    std::vector<float> init(SS_MLP_PARAMS);
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (h_init) memcpy(init.data(), h_init, SS_MLP_PARAMS * sizeof(float));
        else if (g_model.ready) init = g_model.params;
        else return SS_ERR_NO_SELECTOR;
    }
    double total = 0.0;
    for (long i = 0; i < (long)rows * SS_MLP_OUT; ++i) total += h_m[i];
    if (!(total > 0.0)) return -3;
    // The model's bookkeeping from the training rows: configurations with a
    // target per (op, mode), largest batch per (op, size bin, mode).
    int cc[kOps * kSelModes] = {}, bm[kOps * SS_NUM_BINS * kSelModes] = {};
    for (int r = 0; r < rows; ++r) {
        const float *x = h_x + (long)r * SS_MLP_IN;
        const int op = (int)(std::max_element(x, x + 3) - x);
        const int mi = (int)(std::max_element(x + 5, x + 5 + kSelModes) - (x + 5));
        for (int c = SS_MLP_OUT - 1; c >= 0; --c)
            if (h_m[(long)r * SS_MLP_OUT + c] > 0.0f) {
                cc[op * kSelModes + mi] = std::max(cc[op * kSelModes + mi], c + 1);
                break;
            }
        const int n = (int)llround(exp2((double)x[3] * 9.0)), b = (int)llround(exp2((double)x[4] * 14.0));
        const int k = std::min(host_bin(n), SS_NUM_BINS - 1);
        int &slot = bm[(op * SS_NUM_BINS + k) * kSelModes + mi];
        slot = std::max(slot, b);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    size_t wb = 0;
    ss_mlp_workspace_size(rows, &wb);
    const size_t np = SS_MLP_PARAMS * sizeof(float);
    const size_t nx = (size_t)rows * SS_MLP_IN * sizeof(float), nt = (size_t)rows * SS_MLP_OUT * sizeof(float);
    char *buf = nullptr;
    const size_t bytes = 4 * np + nx + 2 * nt + (size_t)steps * sizeof(float) + wb + 8 * 256;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return SS_ERR_CUDA;
    size_t off = 0;
    auto carve = [&](size_t n) { char *p = buf + off; off += (n + 255) / 256 * 256; return p; };
    float *P = (float *)carve(np), *G = (float *)carve(np), *M1 = (float *)carve(np), *M2 = (float *)carve(np);
    float *X = (float *)carve(nx), *T = (float *)carve(nt), *Mk = (float *)carve(nt);
    float *hist = (float *)carve((size_t)steps * sizeof(float));
    void *W = carve(wb);
    int rc = 0;
    if (cudaMemcpyAsync(P, init.data(), np, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(X, h_x, nx, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(T, h_t, nt, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(Mk, h_m, nt, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(M1, 0, np, st) != cudaSuccess || cudaMemsetAsync(M2, 0, np, st) != cudaSuccess)
        rc = SS_ERR_CUDA;
    for (int s = 1; rc == 0 && s <= steps; ++s) {
        if (ss_mlp_grad(P, rows, X, T, Mk, (float)total, G, hist + (s - 1), W, wb, stream) != 0 ||
            ss_mlp_adam(P, G, M1, M2, s, lr, 0.9f, 0.999f, 1e-8f, stream) != 0)
            rc = SS_ERR_CUDA;
    }
    std::vector<float> trained(SS_MLP_PARAMS);
    if (rc == 0 && (cudaMemcpyAsync(trained.data(), P, np, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    (h_loss && cudaMemcpyAsync(h_loss, hist, (size_t)steps * sizeof(float), cudaMemcpyDeviceToHost,
                                               st) != cudaSuccess)))
        rc = SS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = SS_ERR_CUDA;
    cudaFree(buf);
    if (rc != 0) return rc;
    return ss_selector_set(trained.data(), cc, bm);
}

int ss_autotune(int op, int mode, int batch, int max_n, const int *d_n, const double *const *d_A, const int *d_lda,
                const double *const *d_B, const int *d_ldb, const double *const *d_C, const int *d_ldc,
                double *const *d_X, const int *d_ldx, int *d_info, void *d_work, size_t work_bytes, int reps,
                float *h_ms, int *h_bad, int *best_cfg, void *stream)
{
    if (op < 0 || op >= kOps) return -1;
    if (mode == SS_MODE_AUTO || config_count(op, mode) <= 0) return -2;
    if (batch < 1) return -3;
    if (reps < 1) return -17;
    if (!h_ms) return -18;
    if (!best_cfg) return -20;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto call = [&](int cfg) {
        if (op == SS_OP_POTRF)
            return potrf_upper(batch, max_n, d_n, d_A, d_lda, d_X, d_ldx, d_info, mode, cfg, d_work, work_bytes, stream);
        if (op == SS_OP_TRSYL)
            return trsyl_lu(batch, max_n, d_n, d_A, d_lda, d_B, d_ldb, d_C, d_ldc, d_X, d_ldx, d_info, mode, cfg, d_work,
                            work_bytes, stream);
        return trlyap_l(batch, max_n, d_n, d_A, d_lda, d_C, d_ldc, d_X, d_ldx, d_info, mode, cfg, d_work, work_bytes,
                        stream);
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SS_ERR_CUDA; }
    std::vector<int> info(batch);
    const int ncfg = config_count(op, mode);
    int rc = 0, best = -1;
    for (int cfg = 0; cfg < ncfg && rc == 0; ++cfg) {
        int r = call(cfg);                            // warm-up, and the argument check
        if (r != 0) { rc = r; break; }
        std::vector<float> ts;
        for (int i = 0; i < reps; ++i) {
            if (cudaEventRecord(e0, st) != cudaSuccess || call(cfg) != 0 || cudaEventRecord(e1, st) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess) {
                rc = SS_ERR_CUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ts.push_back(ms);
        }
        if (rc != 0) break;
        std::sort(ts.begin(), ts.end());
        h_ms[cfg] = ts[ts.size() / 2];
        if (cudaMemcpyAsync(info.data(), d_info, (size_t)batch * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = SS_ERR_CUDA;
            break;
        }
        const int bad = (int)std::count_if(info.begin(), info.end(), [](int v) { return v != 0; });
        if (h_bad) h_bad[cfg] = bad;
        if (bad == 0 && (best < 0 || h_ms[cfg] < h_ms[best])) best = cfg;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best_cfg = best;
    return rc;
}

}  // extern "C"
