// Planner: picks driver, block size nb and recursion depth for a shape.
//
// Without a cost model the built-in default is used (recursive halving to
// leaves of ~512 rows, blocked leaves with nb = 64).  With a model loaded
// (gb_plan_set_model) every candidate of the standard set is scored by the
// cost-model network on the GPU (one inference launch over all candidates)
// and the argmin of the predicted time is taken; the choice is cached per
// shape.  The network replaces the paper's analytical models (Section V-A:
// Comp(i), and the rule 2 TS(i+1) < TS(i) for the refinement level).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include "common.cuh"
#include "plan.cuh"

namespace gb {

int mlp_forward(const float *P, int D, const float *X, int64_t n, float *Y, float *Z, cudaStream_t s);

namespace {

constexpr int kFeat = 17;
const int kNbs[6] = {16, 32, 64, 128, 256, 512};

gb_plan default_plan(int dtype, int64_t k)
{
    (void)dtype;
    gb_plan p;
    p.reserved = 0;
    p.nb = 64;
    if (k <= 512) {
        p.driver = GB_DRIVER_BLOCKED;
        p.depth = 0;
        return p;
    }
    int d = 0;
    while ((k >> (d + 1)) >= 512 && d < 8) d++;
    p.driver = GB_DRIVER_RECURSIVE;
    p.depth = d;
    return p;
}

struct Model {
    bool loaded = false;
    int D = 0;
    float mean = 0, scale = 1;
    std::vector<float> host;
    float *dparams = nullptr, *dX = nullptr, *dY = nullptr;
    int dev = -1;
    std::map<std::tuple<int, int, int, int, int64_t, int64_t>, std::pair<gb_plan, double>> cache;
};
Model g_model;
std::mutex g_mu;

}  // namespace

int plan_candidates(int dtype, gb_plan *out, int cap)
{
    std::vector<gb_plan> c;
    for (int nb : kNbs) c.push_back({GB_DRIVER_BLOCKED, nb, 0, 0});
    for (int nb : kNbs) c.push_back({GB_DRIVER_ITERATIVE, nb, 0, 0});
    for (int nb : kNbs)
        for (int d = 1; d <= 6; d++) c.push_back({GB_DRIVER_RECURSIVE, nb, d, 0});
    (void)dtype;
    const int n = int(c.size());
    for (int i = 0; i < n && i < cap; i++) out[i] = c[i];
    return n;
}

void plan_features(int dtype, int side, int uplo, int trans, int64_t m, int64_t n, const gb_plan &p, float *f)
{
    for (int i = 0; i < kFeat; i++) f[i] = 0.f;
    f[0] = float(std::log2(double(m > 0 ? m : 1)) / 16.0);
    f[1] = float(std::log2(double(n > 0 ? n : 1)) / 16.0);
    f[2 + (side ? 1 : 0)] = 1.f;
    f[4 + (uplo ? 1 : 0)] = 1.f;
    f[6 + (trans ? 1 : 0)] = 1.f;
    if (dtype >= 0 && dtype < 4) f[8 + dtype] = 1.f;
    f[12] = float(std::log2(double(p.nb > 0 ? p.nb : 1)) / 9.0);
    f[13] = float(p.depth) / 6.f;
    const int drv = p.driver == GB_DRIVER_BLOCKED ? 0 : (p.driver == GB_DRIVER_RECURSIVE ? 1 : 2);
    f[14 + drv] = 1.f;
}

// Score all candidates with the model; returns 0 and the argmin, or an error.
static int model_choose(int dtype, int side, int uplo, int trans, int64_t m, int64_t n, gb_plan *best, double *ms)
{
    const auto key = std::make_tuple(dtype, side, uplo, trans, m, n);
    auto it = g_model.cache.find(key);
    if (it != g_model.cache.end()) {
        *best = it->second.first;
        if (ms) *ms = it->second.second;
        return 0;
    }
    gb_plan cand[64];
    const int nc = plan_candidates(dtype, cand, 64);
    std::vector<float> feats(size_t(nc) * kFeat), pred(nc);
    for (int i = 0; i < nc; i++) plan_features(dtype, side, uplo, trans, m, n, cand[i], &feats[size_t(i) * kFeat]);
    GB_CUDA(cudaMemcpy(g_model.dX, feats.data(), feats.size() * sizeof(float), cudaMemcpyHostToDevice));
    GB_TRY(mlp_forward(g_model.dparams, g_model.D, g_model.dX, nc, g_model.dY, nullptr, 0));
    GB_CUDA(cudaMemcpy(pred.data(), g_model.dY, nc * sizeof(float), cudaMemcpyDeviceToHost));
    int bi = 0;
    for (int i = 1; i < nc; i++)
        if (pred[i] < pred[bi]) bi = i;
    *best = cand[bi];
    const double t = std::exp(double(pred[bi]) * g_model.scale + g_model.mean);
    if (ms) *ms = t;
    g_model.cache[key] = {cand[bi], t};
    return 0;
}

gb_plan choose_plan(int dtype, int side, int uplo, int trans, int64_t m, int64_t n)
{
    const int64_t k = side == GB_LEFT ? m : n;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        int dev = -1;
        cudaGetDevice(&dev);
        if (g_model.loaded && dev == g_model.dev) {
            gb_plan p;
            if (model_choose(dtype, side, uplo, trans, m, n, &p, nullptr) == 0) return p;
        }
    }
    return default_plan(dtype, k);
}

}  // namespace gb

extern "C" {

int gb_plan_candidates(int dtype, gb_plan *out, int cap)
{
    if (dtype < 0 || dtype > 3) return -1;
    if (cap < 0 || (cap > 0 && !out)) return -2;
    return gb::plan_candidates(dtype, out, cap);
}

int gb_plan_features(int dtype, int side, int uplo, int trans, int64_t m, int64_t n, const gb_plan *plan,
                     float *features)
{
    if (!plan) return -7;
    if (!features) return -8;
    gb::plan_features(dtype, side, uplo, trans, m, n, *plan, features);
    return gb::kFeat;
}

int gb_plan_set_model(const char *path)
{
    std::lock_guard<std::mutex> lk(gb::g_mu);
    auto &M = gb::g_model;
    if (!path) {  // unload
        M.loaded = false;
        M.cache.clear();
        return 0;
    }
    FILE *f = std::fopen(path, "rb");
    if (!f) return -1;
    char magic[8];
    int32_t hdr[3];
    float norm[2];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "GBMLP001", 8) == 0 &&
              std::fread(hdr, 4, 3, f) == 3 && std::fread(norm, 4, 2, f) == 2;
    if (!ok || hdr[0] != gb::kFeat || hdr[1] != 64 || hdr[2] <= 0 || hdr[2] > (1 << 20)) {
        std::fclose(f);
        return -1;
    }
    std::vector<float> p(hdr[2]);
    ok = std::fread(p.data(), 4, p.size(), f) == p.size();
    std::fclose(f);
    if (!ok) return -1;
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (M.dev != dev || !M.dparams) {
        if (M.dparams) cudaFree(M.dparams);
        if (M.dX) cudaFree(M.dX);
        if (M.dY) cudaFree(M.dY);
        GB_CUDA(cudaMalloc(&M.dparams, sizeof(float) * (1 << 20)));
        GB_CUDA(cudaMalloc(&M.dX, sizeof(float) * 64 * gb::kFeat));
        GB_CUDA(cudaMalloc(&M.dY, sizeof(float) * 64));
        M.dev = dev;
    }
    GB_CUDA(cudaMemcpy(M.dparams, p.data(), p.size() * sizeof(float), cudaMemcpyHostToDevice));
    M.host = p;
    M.D = hdr[0];
    M.mean = norm[0];
    M.scale = norm[1];
    M.cache.clear();
    M.loaded = true;
    return 0;
}

// The mixed-precision candidates of the precision decision: (low precision,
// leaf order of its recursive low-precision solve), encoded for the network
// as a recursive plan with nb = leaf and depth = log2(kp / leaf) (clamped to
// 0..6), with the BF16-mixed / FP8-mixed dtype one-hot.
static const int kMixedCand[5][2] = {{GB_PREC_BF16, 512}, {GB_PREC_BF16, 1024}, {GB_PREC_BF16, 2048},
                                     {GB_PREC_FP8, 128}, {GB_PREC_FP8, 512}};

int gb_plan_mixed_candidates(int64_t k, int *prec, int64_t *leaf, gb_plan *plans, int cap)
{
    if (k < 0) return -1;
    if (cap < 0) return -5;
    const int64_t kp = (k + 127) / 128 * 128;
    int i = 0;
    for (; i < 5 && i < cap; i++) {
        const int64_t lf = kMixedCand[i][1];
        int d = 0;
        while (d < 6 && (lf << (d + 1)) <= kp) d++;
        if (prec) prec[i] = kMixedCand[i][0];
        if (leaf) leaf[i] = lf;
        if (plans) plans[i] = {GB_DRIVER_RECURSIVE, int(lf), d, 0};
    }
    return 5;
}

int gb_plan_choose_precision(int side, int uplo, int trans, int64_t m, int64_t n, int *prec_out, int64_t *leaf_out,
                             gb_plan *plan_out, double *predicted_ms)
{
    if (side != GB_LEFT && side != GB_RIGHT) return -1;
    if (uplo != GB_LOWER && uplo != GB_UPPER) return -2;
    if (trans != GB_NOTRANS && trans != GB_TRANS) return -3;
    if (m < 0) return -4;
    if (n < 0) return -5;
    if (!prec_out || !leaf_out) return -6;
    std::lock_guard<std::mutex> lk(gb::g_mu);
    const int64_t k = side == GB_LEFT ? m : n;
    if (!gb::g_model.loaded) {
        *prec_out = -1;
        *leaf_out = 0;
        if (plan_out) *plan_out = gb::default_plan(0, k);
        if (predicted_ms) *predicted_ms = -1.0;
        return GB_STATUS_NO_MODEL;
    }
    gb_plan best_plain;
    double t_plain = 0;
    GB_TRY(gb::model_choose(0, side, uplo, trans, m, n, &best_plain, &t_plain));
    int prec[5];
    int64_t leaf[5];
    gb_plan cand[5];
    gb_plan_mixed_candidates(k, prec, leaf, cand, 5);
    float feats[5 * gb::kFeat], pred[5];
    for (int i = 0; i < 5; i++)
        gb::plan_features(prec[i] == GB_PREC_BF16 ? gb::GB_DTYPE_BF16_MIXED : gb::GB_DTYPE_FP8_MIXED, side, uplo,
                          trans, m, n, cand[i], &feats[i * gb::kFeat]);
    GB_CUDA(cudaMemcpy(gb::g_model.dX, feats, sizeof(feats), cudaMemcpyHostToDevice));
    GB_TRY(gb::mlp_forward(gb::g_model.dparams, gb::g_model.D, gb::g_model.dX, 5, gb::g_model.dY, nullptr, 0));
    GB_CUDA(cudaMemcpy(pred, gb::g_model.dY, sizeof(pred), cudaMemcpyDeviceToHost));
    int bi = -1;
    double bt = t_plain;
    for (int i = 0; i < 5; i++) {
        const double t = std::exp(double(pred[i]) * gb::g_model.scale + gb::g_model.mean);
        if (t < bt) {
            bt = t;
            bi = i;
        }
    }
    *prec_out = bi < 0 ? -1 : prec[bi];
    *leaf_out = bi < 0 ? 0 : leaf[bi];
    if (plan_out) *plan_out = bi < 0 ? best_plain : cand[bi];
    if (predicted_ms) *predicted_ms = bt;
    return 0;
}

int gb_plan_choose(int dtype, int side, int uplo, int trans, int64_t m, int64_t n, gb_plan *plan_out,
                   double *predicted_ms)
{
    if (dtype < 0 || dtype > 3) return -1;
    if (side != GB_LEFT && side != GB_RIGHT) return -2;
    if (uplo != GB_LOWER && uplo != GB_UPPER) return -3;
    if (trans != GB_NOTRANS && trans != GB_TRANS) return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    if (!plan_out) return -7;
    std::lock_guard<std::mutex> lk(gb::g_mu);
    if (!gb::g_model.loaded) {
        *plan_out = gb::default_plan(dtype, side == GB_LEFT ? m : n);
        if (predicted_ms) *predicted_ms = -1.0;
        return GB_STATUS_NO_MODEL;
    }
    return gb::model_choose(dtype, side, uplo, trans, m, n, plan_out, predicted_ms);
}

}  // extern "C"
