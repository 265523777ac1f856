// Host plan layer and C ABI (see include/fdas.h for the contract of each entry point).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "fdas_internal.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? FDAS_ERR_OOM : FDAS_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

#define FDAS_CUDA_TRY(call, what)                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
cudaError_t g_encode_err = cudaSuccess;

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    std::call_once(g_encode_once, [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        g_encode_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (g_encode_err == cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode;
}

// 1-D tiled tensor map over n complex64 values (8-byte elements), 256-element boxes.
int encode_input_map(CUtensorMap *map, const void *in, int64_t n)
{
    auto enc = tensor_map_encoder();
    if (!enc) return fail(FDAS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable (%s)", cudaGetErrorString(g_encode_err));
    cuuint64_t dims[1] = {(cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)n * 8};   // unused for rank 1
    cuuint32_t box[1] = {256};
    cuuint32_t estr[1] = {1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 1, const_cast<void *>(in), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(FDAS_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return FDAS_OK;
}

constexpr int kMaxChunks = 8;

}  // namespace

struct fdas_plan_s {
    int device = -1;
    int64_t n_max = 0;
    int M = 0, K_user = 0, K = 0, L = 0, S = 0, G = 0, precision = 0;
    int g_auto = 0;             // 1: templates per block chosen per call from the segment count
    float2 *d_tw = nullptr;     // [L] FP32 twiddles
    double2 *d_tw64 = nullptr;  // [L] FP64 twiddles
    float4 *d_H = nullptr;      // [M][8][L/16] pre-transformed templates
    unsigned char *d_wtc = nullptr;   // tensor-core form: real 32x32 DFT matrices (hi/lo fp16)
    unsigned char *d_tc2c = nullptr;  // two-stage tensor-core form: DFT matrices and twiddles
    unsigned char *d_H16 = nullptr;   // two-stage tensor-core form: fp16 template spectra
    int eH = 0;                       // their power-of-two scale
    float2 *d_h32 = nullptr;          // raw templates [M][K] (time-domain form)
    // grouped plans: templates permuted into support groups, stored shifted to their first tap
    struct Group {
        int first, count, K, S;
        int64_t min_shift;
    };
    int ngroups = 1;
    Group groups[8] = {};
    int *d_rows = nullptr;            // [M] plane row of permuted template r
    int *d_shifts = nullptr;          // [M] first nonzero tap of permuted template r
    int *d_status = nullptr;
    int64_t device_bytes = 0;
    // batched form: the resolved persistent kernel and the plan's own lane
    std::mutex batch_mu;
    fdas::BatchKernel bk;
    int bk_version = 0;                     // bumped whenever bk changes (graphs must be rebuilt)
    fdas::Lane lane0;
    // autotuner results, ms per proxy batch, [L index][G index: per call, 5, 17, 85], and the
    // two-stage tensor-core form
    float tune_ms[3][4] = {};
    float tune_ms_tc = 0.f;
    int tuned = 0;
    // host-buffer entry point
    std::mutex host_mu;
    void *d_in_stage = nullptr;
    float *d_out_stage = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t chunk_ev[kMaxChunks] = {};
};

namespace {

void plan_free(fdas_plan p)
{
    if (!p) return;
    DeviceGuard g(p->device);
    cudaFree(p->d_tw);
    cudaFree(p->d_tw64);
    cudaFree(p->d_H);
    cudaFree(p->d_wtc);
    cudaFree(p->d_tc2c);
    cudaFree(p->d_H16);
    cudaFree(p->d_h32);
    cudaFree(p->d_rows);
    cudaFree(p->d_shifts);
    cudaFree(p->d_status);
    cudaFree(p->d_in_stage);
    cudaFree(p->d_out_stage);
    fdas::lane_free(&p->lane0);
    for (auto &e : p->chunk_ev)
        if (e) cudaEventDestroy(e);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    delete p;
}

int validate_convolve(fdas_plan p, const void *in, int64_t n, const float *out)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    if (!in || !out) return fail(FDAS_ERR_INVALID_ARG, "null input or output pointer");
    if (n < 1 || n > p->n_max) return fail(FDAS_ERR_INVALID_ARG, "n=%lld outside [1, n_max=%lld]", (long long)n, (long long)p->n_max);
    if (reinterpret_cast<uintptr_t>(in) % 16) return fail(FDAS_ERR_INVALID_ARG, "input pointer must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(out) % 4) return fail(FDAS_ERR_INVALID_ARG, "output pointer must be 4-byte aligned");
    const uintptr_t i0 = reinterpret_cast<uintptr_t>(in), i1 = i0 + (uintptr_t)n * 8;
    const uintptr_t o0 = reinterpret_cast<uintptr_t>(out), o1 = o0 + (uintptr_t)n * 4 * (uintptr_t)p->M;
    if (i0 < o1 && o0 < i1) return fail(FDAS_ERR_INVALID_ARG, "input and output overlap");
    return FDAS_OK;
}

int64_t n_segments(const fdas_plan p, int64_t n) { return (n + p->S - 1) / p->S; }

// Templates per block for a launch over `nseg` segments of `m` templates.  A plan with a
// fixed G keeps it.  Otherwise the templates are split into ng groups so that short arrays
// still fill the GPU: ng = (4 * resident blocks / nseg)^0.7, rounded, between 1 and m/5.
// One group per block costs a forward FFT and the segment load; the exponent and the
// limit of five templates per block were fitted to measured times for 2^14..2^22 points
// and 85 templates (a full-size array keeps all templates in one block).
int call_G(const fdas_plan p, int64_t nseg, int m)
{
    if (!p->g_auto) return std::min(p->G, m);
    const int slots = std::max(1, p->bk.resident);
    const double r = 4.0 * slots / (double)std::max<int64_t>(1, nseg);
    int ng = (int)std::lround(std::pow(r, 0.7));
    ng = std::max(1, std::min(ng, std::max(1, m / 5)));
    return (m + ng - 1) / ng;
}

fdas::OlsArgs base_args(fdas_plan p, int64_t n, float *out)
{
    fdas::OlsArgs a;
    a.H = p->d_H;
    a.tw = p->d_tw;
    a.out = out;
    a.n = n;
    a.M = p->M;
    a.G = call_G(p, n_segments(p, n), p->M);
    a.S = p->S;
    a.K = p->K;
    a.seg_begin = 0;
    a.status = p->d_status;
    return a;
}

// Launch segments [s0, s1) of an ungrouped plan (a carries the epilogue settings).
int launch_range(fdas_plan p, const CUtensorMap *map, fdas::OlsArgs a, int64_t s0, int64_t s1, cudaStream_t stream)
{
    a.seg_begin = (int)s0;
    cudaError_t e = fdas::launch_ols_fp32(p->L, map, a, (int)(s1 - s0), stream);
    if (e != cudaSuccess) return cuda_fail(e, "segment kernel launch");
    return FDAS_OK;
}

// All segments of every template group: one launch per group.
int launch_all(fdas_plan p, const CUtensorMap *map, const fdas::OlsArgs &a0, int64_t n, cudaStream_t stream)
{
    if (p->ngroups <= 1 && !p->d_rows) return launch_range(p, map, a0, 0, n_segments(p, n), stream);
    for (int g = 0; g < p->ngroups; ++g) {
        const auto &gr = p->groups[g];
        fdas::OlsArgs a = a0;
        a.H = p->d_H + (size_t)gr.first * 8 * (p->L / 16);
        a.M = gr.count;
        a.S = gr.S;
        a.K = gr.K;
        a.rows = p->d_rows + gr.first;
        a.shifts = p->d_shifts + gr.first;
        const int64_t span = n - gr.min_shift;
        const int64_t nseg = span > 0 ? (span + gr.S - 1) / gr.S : 1;   // one segment writes the zero prefix
        a.G = call_G(p, nseg, gr.count);
        cudaError_t e = fdas::launch_ols_fp32(p->L, map, a, (int)nseg, stream);
        if (e != cudaSuccess) return cuda_fail(e, "segment kernel launch (template group)");
    }
    return FDAS_OK;
}

int enqueue_segments(fdas_plan p, const CUtensorMap *map, int64_t n, float *out, int64_t s0, int64_t s1,
                     cudaStream_t stream)
{
    const fdas::OlsArgs a = base_args(p, n, out);
    if (p->precision == FDAS_PREC_TC_FP16) {
        fdas::OlsArgs b = a;
        b.seg_begin = (int)s0;
        cudaError_t e = fdas::launch_ols_tc(map, b, p->d_wtc, (int)(s1 - s0), stream);
        if (e != cudaSuccess) return cuda_fail(e, "segment kernel launch");
        return FDAS_OK;
    }
    if (p->precision == FDAS_PREC_TC_DFT2) {
        fdas::OlsArgs b = a;
        b.seg_begin = (int)s0;
        cudaError_t e = fdas::launch_ols_tc2(map, b, p->d_H16, p->d_tc2c, p->eH, (int)(s1 - s0), stream);
        if (e != cudaSuccess) return cuda_fail(e, "segment kernel launch (two-stage tensor-core form)");
        return FDAS_OK;
    }
    return launch_range(p, map, a, s0, s1, stream);
}

// Support of each template (first and last nonzero tap), the grouping that minimises the
// number of L-point transforms for arrays of n_ref points (equal-count groups of templates
// sorted by support length, 1 to 6 groups), and the permuted, shifted template array.
int plan_groups(fdas_plan p, const float2 *h_host, int64_t n_ref, std::vector<float2> &shifted,
                std::vector<int> &rows, std::vector<int> &shifts)
{
    const int M = p->M, K = p->K_user, L = p->L;
    std::vector<int> first(M), len(M);
    for (int z = 0; z < M; ++z) {
        int a = -1, b = -1;
        for (int k = 0; k < K; ++k) {
            const float2 v = h_host[(size_t)z * K + k];
            if (v.x != 0.f || v.y != 0.f) {
                if (a < 0) a = k;
                b = k;
            }
        }
        first[z] = a < 0 ? 0 : a;
        len[z] = a < 0 ? 1 : b - a + 1;
    }
    std::vector<int> order(M);
    for (int z = 0; z < M; ++z) order[z] = z;
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return len[u] < len[v]; });
    auto frame = [](int k) { return 4 * ((k - 1 + 3) / 4) + 1; };
    double best = 1e300;
    int best_ng = 1;
    for (int ng = 1; ng <= std::min(6, M); ++ng) {
        double cost = 0;
        for (int g = 0; g < ng; ++g) {
            const int lo = (int)((int64_t)M * g / ng), hi = (int)((int64_t)M * (g + 1) / ng);
            if (hi <= lo) continue;
            const int Kg = frame(len[order[hi - 1]]), Sg = L - Kg + 1;
            cost += (double)((n_ref + Sg - 1) / Sg) * (hi - lo + 1);
        }
        if (cost < best * (1.0 - 1e-9)) {
            best = cost;
            best_ng = ng;
        }
    }
    p->ngroups = best_ng;
    for (int g = 0; g < best_ng; ++g) {
        const int lo = (int)((int64_t)M * g / best_ng), hi = (int)((int64_t)M * (g + 1) / best_ng);
        auto &gr = p->groups[g];
        gr.first = lo;
        gr.count = hi - lo;
        gr.K = frame(len[order[hi - 1]]);
        gr.S = L - gr.K + 1;
        gr.min_shift = INT64_MAX;
        for (int r = lo; r < hi; ++r) gr.min_shift = std::min<int64_t>(gr.min_shift, first[order[r]]);
    }
    shifted.assign((size_t)M * K, make_float2(0.f, 0.f));
    rows.resize(M);
    shifts.resize(M);
    for (int r = 0; r < M; ++r) {
        const int z = order[r];
        rows[r] = z;
        shifts[r] = first[z];
        for (int k = 0; k < len[z]; ++k) shifted[(size_t)r * K + k] = h_host[(size_t)z * K + first[z] + k];
    }
    return FDAS_OK;
}

// (Re)build the FP64 twiddles and the pre-transformed templates for segment length L.
int build_templates(fdas_plan p, const float2 *d_h32, int L)
{
    cudaFree(p->d_tw);
    cudaFree(p->d_tw64);
    cudaFree(p->d_H);
    p->d_tw = nullptr;
    p->d_tw64 = nullptr;
    p->d_H = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_tw, sizeof(float2) * L)) != cudaSuccess) return cuda_fail(e, "cudaMalloc twiddles");
    if ((e = cudaMalloc(&p->d_tw64, sizeof(double2) * L)) != cudaSuccess) return cuda_fail(e, "cudaMalloc twiddles64");
    if ((e = cudaMalloc(&p->d_H, sizeof(float4) * (size_t)p->M * 8 * (L / 16))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc templates");
    if ((e = fdas::launch_twiddles(L, p->d_tw64, p->d_tw, nullptr)) != cudaSuccess) return cuda_fail(e, "twiddle kernel");
    if ((e = fdas::launch_pretransform(L, d_h32, p->M, p->K_user, p->d_tw64, p->d_H,
                                        p->precision == FDAS_PREC_TC_FP16, nullptr)) != cudaSuccess)
        return cuda_fail(e, "pretransform kernel");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "plan-time kernels");
    p->L = L;
    p->S = (L - p->K + 1) & ~3;
    p->bk = fdas::BatchKernel();
    p->bk_version++;
    if ((e = fdas::batch_kernel(L, &p->bk)) != cudaSuccess) return cuda_fail(e, "batch kernel attributes");
    if (p->precision == FDAS_PREC_TC_DFT2 && (e = fdas::tc2_batch_kernel(&p->bk)) != cudaSuccess)
        return cuda_fail(e, "tensor-core batch kernel attributes");
    return FDAS_OK;
}

int validate_batch(fdas_plan p, int count, const void *const *ins, const int64_t *ns, float *const *outs)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    if (p->d_rows) return fail(FDAS_ERR_UNSUPPORTED, "the batched forms are built for ungrouped plans");
    if (p->precision == FDAS_PREC_TC_FP16)
        return fail(FDAS_ERR_UNSUPPORTED, "the batched forms are not built for the single-pass tensor-core form");
    if (count < 0 || (count > 0 && (!ins || !ns || !outs))) return fail(FDAS_ERR_INVALID_ARG, "bad batch arrays");
    for (int i = 0; i < count; ++i) {
        int rc = validate_convolve(p, ins[i], ns[i], outs[i]);
        if (rc) return fail(rc, "batch entry %d: %s", i, g_last_error.c_str());
    }
    return FDAS_OK;
}

int enqueue_batch(fdas_plan p, int count, const void *const *ins, const int64_t *ns, float *const *outs,
                  cudaStream_t stream)
{
    return fdas::lane_launch(p, &p->lane0, count, ins, ns, outs, stream);
}

// Autotuner: time the persistent batch kernel for every (L, G) candidate -- G = 0 being the
// per-call choice -- and, with mode 2, the two-stage tensor-core form (L = 2048), on a seeded
// proxy of the batches the plan will serve: 16 arrays with lengths log-uniform in [n_min,
// n_max]; keep the fastest.  Results are cached per process by (device, M, K, n_min, n_max,
// mode, fixed G).
struct TuneKey {
    int dev, M, K, mode, fixed_G;
    int64_t n_min, n_max;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(dev, M, K, mode, fixed_G, n_min, n_max) < std::tie(o.dev, o.M, o.K, o.mode, o.fixed_G, o.n_min, o.n_max);
    }
};
struct TuneVal {
    int L, G, precision;
    float ms[3][4], ms_tc;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

const int kTuneL[3] = {1024, 2048, 4096};
const int kTuneG[4] = {0, 5, 17, 85};
constexpr int kTuneArrays = 16;

// Lengths of the proxy batch: log-uniform in [lo, hi] from a fixed splitmix64 sequence.
std::vector<int64_t> tune_lengths(int64_t lo, int64_t hi)
{
    std::vector<int64_t> ns(kTuneArrays);
    uint64_t x = 0x243F6A8885A308D3ull;
    for (auto &n : ns) {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double u = (double)(z >> 11) / 9007199254740992.0;
        n = (int64_t)std::llround(std::exp(std::log((double)lo) + u * (std::log((double)hi) - std::log((double)lo))));
        n = std::max(lo, std::min(hi, n));
    }
    return ns;
}

int tc2_resources(fdas_plan p)   // the two-stage form's constants and fp16 spectra (allocated once)
{
    cudaError_t e;
    if (!p->d_tc2c && (e = cudaMalloc(&p->d_tc2c, fdas::tc2_const_bytes())) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc tensor-core constants");
    if (!p->d_H16 && (e = cudaMalloc(&p->d_H16, fdas::tc2_template_bytes(p->M))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc fp16 template spectra");
    if ((e = fdas::launch_tc2_constants(p->d_tc2c, nullptr)) != cudaSuccess) return cuda_fail(e, "tensor-core constants kernel");
    return FDAS_OK;
}

int autotune(fdas_plan p, const float2 *d_h32, int fixed_G, int mode, int64_t n_min)
{
    const int64_t n_max = p->n_max;
    n_min = n_min > 0 ? std::min(n_min, n_max) : std::max<int64_t>(1, n_max / 16);
    const TuneKey key{p->device, p->M, p->K_user, mode, fixed_G, n_min, n_max};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p->L = it->second.L;
            p->G = it->second.G ? it->second.G : p->M;
            p->g_auto = it->second.G == 0;
            p->precision = it->second.precision;
            std::memcpy(p->tune_ms, it->second.ms, sizeof p->tune_ms);
            p->tune_ms_tc = it->second.ms_tc;
            p->tuned = 1;
            return p->precision == FDAS_PREC_TC_DFT2 ? tc2_resources(p) : FDAS_OK;
        }
    }
    const std::vector<int64_t> ns = tune_lengths(n_min, n_max);
    void *d_in = nullptr;
    float *d_out = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&d_in, sizeof(float2) * n_max)) != cudaSuccess) return cuda_fail(e, "autotune input");
    if ((e = cudaMalloc(&d_out, sizeof(float) * n_max * p->M)) != cudaSuccess) {
        cudaFree(d_in);
        return cuda_fail(e, "autotune output");
    }
    cudaMemset(d_in, 0x3c, sizeof(float2) * n_max);   // finite, non-denormal values
    // every proxy array reads a prefix of one input and writes one shared plane buffer: only
    // the time is kept
    std::vector<const void *> ins(kTuneArrays, d_in);
    std::vector<float *> outs(kTuneArrays, d_out);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bestL = p->L, bestG = p->G, bestP = FDAS_PREC_FP32, rc = FDAS_OK;
    auto time_batch = [&](float *out_ms) {
        float ms = 0.f;
        for (int rep = 0; rep < 4 && rc == FDAS_OK; ++rep) {
            cudaEventRecord(e0, nullptr);
            rc = enqueue_batch(p, kTuneArrays, ins.data(), ns.data(), outs.data(), nullptr);
            cudaEventRecord(e1, nullptr);
            if (rc == FDAS_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_fail(e, "autotune run");
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t / 3.f;
        }
        *out_ms = ms;
    };
    for (int li = 0; li < 3 && rc == FDAS_OK; ++li) {
        const int L = kTuneL[li];
        if (p->K > L - 4) continue;
        p->precision = FDAS_PREC_FP32;
        if ((rc = build_templates(p, d_h32, L))) break;
        for (int gi = 0; gi < 4 && rc == FDAS_OK; ++gi) {
            const int G = fixed_G ? fixed_G : std::min(kTuneG[gi], p->M);
            p->g_auto = G == 0;
            p->G = G ? G : p->M;
            float ms = 0.f;
            time_batch(&ms);
            p->tune_ms[li][gi] = ms;
            if (rc == FDAS_OK && ms < best) {
                best = ms;
                bestL = L;
                bestG = G;
                bestP = FDAS_PREC_FP32;
            }
            if (fixed_G) break;
        }
    }
    if (rc == FDAS_OK && mode == 2 && p->K <= 2048 - 4) {   // the two-stage tensor-core form
        p->precision = FDAS_PREC_TC_DFT2;
        p->g_auto = 0;
        p->G = p->M;
        if (!(rc = tc2_resources(p)) && !(rc = build_templates(p, d_h32, 2048))) {
            if ((e = fdas::launch_tc2_pretransform(d_h32, p->M, p->K_user, p->d_tw64, p->eH, p->d_H16, nullptr)) != cudaSuccess)
                rc = cuda_fail(e, "fp16 template pre-transform");
            float ms = 0.f;
            if (rc == FDAS_OK) time_batch(&ms);
            p->tune_ms_tc = ms;
            if (rc == FDAS_OK && ms < best) {
                best = ms;
                bestL = 2048;
                bestG = 0;
                bestP = FDAS_PREC_TC_DFT2;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_in);
    cudaFree(d_out);
    if (rc != FDAS_OK) return rc;
    if ((rc = fdas_plan_status(p, nullptr)) != FDAS_OK) return rc;
    p->L = bestL;
    p->precision = bestP;
    p->g_auto = bestP == FDAS_PREC_FP32 && bestG == 0;
    p->G = bestG ? bestG : p->M;
    if (bestP != FDAS_PREC_TC_DFT2) {   // the tensor-core candidate's buffers are not kept
        cudaFree(p->d_tc2c);
        cudaFree(p->d_H16);
        p->d_tc2c = nullptr;
        p->d_H16 = nullptr;
    }
    p->tuned = 1;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneVal v{bestL, bestG, bestP, {}, p->tune_ms_tc};
    std::memcpy(v.ms, p->tune_ms, sizeof v.ms);
    g_tune_cache[key] = v;
    return FDAS_OK;
}

}  // namespace

namespace fdas {

// Fill the table and launch arguments of one persistent launch over arrays [first, first + cnt).
// FP32 plans: items (array, template group, segment), G from the total segment count.  Two-stage
// tensor-core plans: items (array, segment pair, template-pair group), the groups per segment
// pair from the total number of segment pairs.
static int fill_batch(fdas_plan p, BatchTable &t, OlsArgs &a, int first, int cnt, const void *const *ins,
                      const int64_t *ns, float *const *outs)
{
    a = OlsArgs();
    a.H = p->d_H;
    a.tw = p->d_tw;
    a.M = p->M;
    a.S = p->S;
    a.K = p->K;
    a.status = p->d_status;
    const bool tc2 = p->precision == FDAS_PREC_TC_DFT2;
    int64_t units = 0;   // segments (FP32) or segment pairs (tensor-core form)
    for (int i = 0; i < cnt; ++i) {
        const int64_t ns_i = n_segments(p, ns[first + i]);
        units += tc2 ? (ns_i + 1) / 2 : ns_i;
    }
    int per_unit;
    if (tc2) {
        a.H16 = p->d_H16;
        a.cst = p->d_tc2c;
        a.eH = p->eH;
        a.ng = 1;   // the kernel shares the launch's (segment pair, template pair) units out evenly
        a.G = p->M;
        per_unit = 1;
    } else {
        a.G = call_G(p, units, p->M);
        per_unit = (p->M + a.G - 1) / a.G;
    }
    int64_t items = 0;
    for (int i = 0; i < cnt; ++i) {
        BatchArray &ar = t.arr[i];
        int rc = encode_input_map(&ar.map, ins[first + i], ns[first + i]);
        if (rc) return rc;
        ar.out = outs[first + i];
        ar.n = ns[first + i];
        ar.nseg = (int)n_segments(p, ar.n);
        ar.item_off = items;
        items += (int64_t)(tc2 ? (ar.nseg + 1) / 2 : ar.nseg) * per_unit;
    }
    if (tc2 && items * ((p->M + 1) / 2) >= ((int64_t)1 << 31))   // the kernel counts units in 32 bits
        return fail(FDAS_ERR_INVALID_ARG, "batch too large for one launch of the tensor-core form");
    t.count = cnt;
    t.total_items = items;
    return FDAS_OK;
}

// Direct (graph-free) launches of the persistent batch kernel, one per table of up to
// kBatchMax arrays; launch c takes its work counter at counters[c].  The counters are
// cleared on `stream` first.  Host memory used: the stack only; no device allocation.
int batch_direct(fdas_plan p, int count, const void *const *ins, const int64_t *ns, float *const *outs,
                 int *counters, int max_chunks, cudaStream_t stream)
{
    int rc = validate_batch(p, count, ins, ns, outs);
    if (rc) return rc;
    const int chunks = (count + kBatchMax - 1) / kBatchMax;
    if (chunks > max_chunks)
        return fail(FDAS_ERR_INVALID_ARG, "batch of %d arrays exceeds the %d-array limit of this entry point", count,
                    max_chunks * kBatchMax);
    if (count == 0) return FDAS_OK;
    cudaError_t e;
    if ((e = cudaMemsetAsync(counters, 0, sizeof(int) * chunks, stream)) != cudaSuccess)
        return cuda_fail(e, "clear work counters");
    BatchTable t;
    OlsArgs a;
    for (int c = 0; c < chunks; ++c) {
        const int first = c * kBatchMax, cnt = std::min(kBatchMax, count - first);
        if ((rc = fill_batch(p, t, a, first, cnt, ins, ns, outs))) return rc;
        int *counter = counters + c;
        void *args[3] = {&t, &a, &counter};
        if ((e = cudaLaunchKernel(p->bk.fn, dim3(p->bk.resident), dim3(p->bk.block), args, p->bk.smem, stream)) !=
            cudaSuccess)
            return cuda_fail(e, "persistent batch kernel launch");
    }
    return FDAS_OK;
}

void lane_free(Lane *l)
{
    if (l->exec) cudaGraphExecDestroy(l->exec);
    if (l->graph) cudaGraphDestroy(l->graph);
    cudaFree(l->d_counter);
    if (l->table) ::operator delete(l->table, std::align_val_t(alignof(BatchTable)));
    *l = Lane();
}

// Build (or rebuild after the plan's kernel changed) the lane's graph:
// [memset work counter] -> [persistent kernel over all resident blocks].
static int lane_ensure(fdas_plan p, Lane *l)
{
    cudaError_t e;
    if (!l->d_counter) {
        if ((e = cudaMalloc(&l->d_counter, 256)) != cudaSuccess) return cuda_fail(e, "cudaMalloc work counter");
        if ((e = cudaMemset(l->d_counter, 0, 256)) != cudaSuccess) return cuda_fail(e, "memset work counter");
    }
    if (!l->table) {
        l->table = static_cast<BatchTable *>(::operator new(sizeof(BatchTable), std::align_val_t(alignof(BatchTable)), std::nothrow));
        if (!l->table) return fail(FDAS_ERR_OOM, "host batch table");
        std::memset(l->table, 0, sizeof(BatchTable));
    }
    if (l->exec && l->version == p->bk_version) return FDAS_OK;
    if (l->exec) cudaGraphExecDestroy(l->exec);
    if (l->graph) cudaGraphDestroy(l->graph);
    l->exec = nullptr;
    l->graph = nullptr;
    if ((e = cudaGraphCreate(&l->graph, 0)) != cudaSuccess) return cuda_fail(e, "graph create");
    cudaMemsetParams mp = {};
    mp.dst = l->d_counter;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 1;
    mp.height = 1;
    cudaGraphNode_t ms;
    if ((e = cudaGraphAddMemsetNode(&ms, l->graph, nullptr, 0, &mp)) != cudaSuccess) return cuda_fail(e, "graph memset node");
    void *args[3] = {l->table, &l->args, &l->d_counter};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void *>(p->bk.fn);
    kp.gridDim = dim3(p->bk.resident);
    kp.blockDim = dim3(p->bk.block);
    kp.sharedMemBytes = (unsigned)p->bk.smem;
    kp.kernelParams = args;
    if ((e = cudaGraphAddKernelNode(&l->kernel_node, l->graph, &ms, 1, &kp)) != cudaSuccess)
        return cuda_fail(e, "graph kernel node");
    if ((e = cudaGraphInstantiate(&l->exec, l->graph, 0)) != cudaSuccess) return cuda_fail(e, "graph instantiate");
    l->version = p->bk_version;
    return FDAS_OK;
}

// Fill the lane's table for arrays [first, first + cnt) and replay its graph on `stream`.
static int lane_chunk(fdas_plan p, Lane *l, int first, int cnt, const void *const *ins, const int64_t *ns,
                      float *const *outs, cudaStream_t stream)
{
    int rc = fill_batch(p, *l->table, l->args, first, cnt, ins, ns, outs);
    if (rc) return rc;
    void *args[3] = {l->table, &l->args, &l->d_counter};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void *>(p->bk.fn);
    kp.gridDim = dim3(p->bk.resident);
    kp.blockDim = dim3(p->bk.block);
    kp.sharedMemBytes = (unsigned)p->bk.smem;
    kp.kernelParams = args;
    cudaError_t e;
    if ((e = cudaGraphExecKernelNodeSetParams(l->exec, l->kernel_node, &kp)) != cudaSuccess)
        return cuda_fail(e, "graph kernel params");
    if ((e = cudaGraphLaunch(l->exec, stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
    return FDAS_OK;
}

int lane_launch(fdas_plan p, Lane *l, int count, const void *const *ins, const int64_t *ns, float *const *outs,
                cudaStream_t stream)
{
    int rc = lane_ensure(p, l);
    if (rc) return rc;
    for (int first = 0; first < count; first += kBatchMax) {
        const int cnt = std::min(kBatchMax, count - first);
        if ((rc = lane_chunk(p, l, first, cnt, ins, ns, outs, stream))) return rc;
    }
    return FDAS_OK;
}

int validate_array(fdas_plan p, const void *in, int64_t n, const float *out)
{
    return validate_convolve(p, in, n, out);
}

int plan_templates(fdas_plan p) { return p ? p->M : 0; }
int plan_grouped(fdas_plan p) { return p && p->d_rows ? 1 : 0; }
int plan_precision(fdas_plan p) { return p ? p->precision : -1; }
int *plan_status_word(fdas_plan p) { return p ? p->d_status : nullptr; }
int64_t plan_n_max(fdas_plan p) { return p ? p->n_max : 0; }

// Plan accessor and error reporting for code outside this file.
int plan_device(fdas_plan p) { return p ? p->device : -1; }
int set_error(int code, const char *msg) { return fail(code, "%s", msg); }

}  // namespace fdas

extern "C" {

const char *fdas_version(void) { return "fdas-gb300 0.1 (sm_103a)"; }

const char *fdas_strerror(int code)
{
    switch (code) {
    case FDAS_OK: return "ok";
    case FDAS_ERR_INVALID_ARG: return "invalid argument";
    case FDAS_ERR_OOM: return "out of memory";
    case FDAS_ERR_CUDA: return "CUDA error";
    case FDAS_ERR_TIMEOUT: return "timed out";
    case FDAS_ERR_BUSY: return "busy";
    case FDAS_ERR_REJECTED: return "rejected";
    case FDAS_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown error";
    }
}

const char *fdas_last_error(void) { return g_last_error.c_str(); }

int fdas_plan_create(fdas_plan *out, int64_t n_max, const void *templates, int M, int K, const fdas_opts *opts)
{
    if (!out) return fail(FDAS_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    fdas_opts o = {};
    if (opts) o = *opts;
    const int L = o.seg_len ? o.seg_len : 2048;
    if (L != 1024 && L != 2048 && L != 4096) return fail(FDAS_ERR_INVALID_ARG, "seg_len %d not in {1024, 2048, 4096}", L);
    if (o.precision != FDAS_PREC_FP32 && o.precision != FDAS_PREC_TC_FP16 && o.precision != FDAS_PREC_TC_DFT2)
        return fail(FDAS_ERR_UNSUPPORTED, "precision %d not built", o.precision);
    if (o.precision != FDAS_PREC_FP32 && (L != 2048 || o.autotune))
        return fail(FDAS_ERR_UNSUPPORTED, "the tensor-core forms are built for seg_len 2048 without autotuning");
    if (!templates) return fail(FDAS_ERR_INVALID_ARG, "null templates");
    if (M < 1) return fail(FDAS_ERR_INVALID_ARG, "n_templates=%d < 1", M);
    if (K < 1 || K > L - 4) return fail(FDAS_ERR_INVALID_ARG, "tpl_len=%d outside [1, %d]", K, L - 4);
    if (n_max < 1 || n_max > (int64_t(1) << 30)) return fail(FDAS_ERR_INVALID_ARG, "n_max=%lld outside [1, 2^30]", (long long)n_max);
    if (o.tpl_per_cta < 0 || o.tpl_per_cta > M) return fail(FDAS_ERR_INVALID_ARG, "tpl_per_cta=%d outside [0, %d]", o.tpl_per_cta, M);
    if (o.group_support != 0 && o.group_support != 1) return fail(FDAS_ERR_INVALID_ARG, "group_support=%d not 0 or 1", o.group_support);
    if (o.autotune < 0 || o.autotune > 2) return fail(FDAS_ERR_INVALID_ARG, "autotune=%d not 0, 1 or 2", o.autotune);
    if (o.tune_n_min < 0) return fail(FDAS_ERR_INVALID_ARG, "tune_n_min=%lld < 0", (long long)o.tune_n_min);
    if (o.group_support && (o.precision != FDAS_PREC_FP32 || o.autotune))
        return fail(FDAS_ERR_UNSUPPORTED, "template groups are built for the FP32 form without autotuning");

    fdas_plan p = new (std::nothrow) fdas_plan_s;
    if (!p) return fail(FDAS_ERR_OOM, "host allocation");
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return fail(FDAS_ERR_CUDA, "no current CUDA device");
    }
    p->n_max = n_max;
    p->M = M;
    p->K_user = K;
    p->K = 4 * ((K - 1 + 3) / 4) + 1;           // frame with K-1 a multiple of 4 (trailing zero taps):
                                                // segment starts and row segments stay 16-byte aligned
    p->L = L;
    p->S = (L - p->K + 1) & ~3;                 // multiple of 4, <= L - K + 1
    p->G = o.tpl_per_cta ? o.tpl_per_cta : M;
    p->precision = o.precision;
    p->g_auto = (o.tpl_per_cta == 0 && !o.autotune && o.precision == FDAS_PREC_FP32) ? 1 : 0;

    auto cleanup_fail = [&](int code) {
        plan_free(p);
        return code;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_status, sizeof(int))) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc status"));
    if ((e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess) return cleanup_fail(cuda_fail(e, "memset status"));
    float2 *d_h32 = nullptr;
    const size_t h_bytes = sizeof(float2) * (size_t)M * K;
    if ((e = cudaMalloc(&d_h32, h_bytes)) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc template staging"));
    if ((e = cudaMemcpy(d_h32, templates, h_bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(d_h32);
        return cleanup_fail(cuda_fail(e, "copy templates"));
    }
    int rc = FDAS_OK;
    if (p->precision == FDAS_PREC_TC_FP16) {
        if ((e = cudaMalloc(&p->d_wtc, fdas::tc_matrix_bytes())) != cudaSuccess) rc = cuda_fail(e, "cudaMalloc DFT matrices");
        else if ((e = fdas::launch_tc_matrices(p->d_wtc, nullptr)) != cudaSuccess) rc = cuda_fail(e, "DFT matrix kernel");
    }
    {   // two-stage tensor-core form's template scale 2^eH: the largest power of two with
        // 2^eH max_z sum_k |h_z[k]| <= 16, which bounds every |FFT(h_z)[f]| 2^eH by 16 (fp16 range)
        const float2 *hh = static_cast<const float2 *>(templates);
        double l1max = 0.0;
        for (int z = 0; z < M; ++z) {
            double l1 = 0.0;
            for (int k = 0; k < K; ++k) l1 += std::hypot((double)hh[(size_t)z * K + k].x, (double)hh[(size_t)z * K + k].y);
            l1max = std::max(l1max, l1);
        }
        p->eH = l1max > 0.0 ? (int)std::floor(std::log2(16.0 / l1max)) : 0;
        p->eH = std::max(-60, std::min(60, p->eH));
    }
    if (rc == FDAS_OK && p->precision == FDAS_PREC_TC_DFT2) rc = tc2_resources(p);
    if (rc == FDAS_OK && o.autotune) rc = autotune(p, d_h32, o.tpl_per_cta, o.autotune, o.tune_n_min);
    p->d_h32 = d_h32;   // kept for the time-domain form
    if (rc == FDAS_OK && o.group_support) {
        // transform the permuted, shifted templates instead of the raw ones
        std::vector<float2> shifted;
        std::vector<int> rows, shifts;
        rc = plan_groups(p, static_cast<const float2 *>(templates), n_max, shifted, rows, shifts);
        float2 *d_hs = nullptr;
        if (rc == FDAS_OK && (e = cudaMalloc(&d_hs, h_bytes)) != cudaSuccess) rc = cuda_fail(e, "cudaMalloc shifted templates");
        if (rc == FDAS_OK && (e = cudaMalloc(&p->d_rows, sizeof(int) * M)) != cudaSuccess) rc = cuda_fail(e, "cudaMalloc rows");
        if (rc == FDAS_OK && (e = cudaMalloc(&p->d_shifts, sizeof(int) * M)) != cudaSuccess) rc = cuda_fail(e, "cudaMalloc shifts");
        if (rc == FDAS_OK && (e = cudaMemcpy(d_hs, shifted.data(), h_bytes, cudaMemcpyHostToDevice)) != cudaSuccess)
            rc = cuda_fail(e, "copy shifted templates");
        if (rc == FDAS_OK && (e = cudaMemcpy(p->d_rows, rows.data(), sizeof(int) * M, cudaMemcpyHostToDevice)) != cudaSuccess)
            rc = cuda_fail(e, "copy rows");
        if (rc == FDAS_OK && (e = cudaMemcpy(p->d_shifts, shifts.data(), sizeof(int) * M, cudaMemcpyHostToDevice)) != cudaSuccess)
            rc = cuda_fail(e, "copy shifts");
        if (rc == FDAS_OK) rc = build_templates(p, d_hs, p->L);
        cudaFree(d_hs);
    } else if (rc == FDAS_OK) {
        rc = build_templates(p, d_h32, p->L);
    }
    if (rc == FDAS_OK && p->precision == FDAS_PREC_TC_DFT2) {
        if ((e = fdas::launch_tc2_pretransform(d_h32, M, K, p->d_tw64, p->eH, p->d_H16, nullptr)) != cudaSuccess)
            rc = cuda_fail(e, "fp16 template pre-transform");
        else if ((e = cudaDeviceSynchronize()) != cudaSuccess) rc = cuda_fail(e, "plan-time kernels");
    }
    if (rc != FDAS_OK) return cleanup_fail(rc);
    p->device_bytes = (int64_t)(sizeof(float2) * p->L + sizeof(double2) * p->L +
                                sizeof(float4) * (size_t)M * 8 * (p->L / 16) + sizeof(int) + h_bytes +
                                (p->d_wtc ? fdas::tc_matrix_bytes() : 0) + (p->d_rows ? 2 * sizeof(int) * M : 0) +
                                (p->d_tc2c ? fdas::tc2_const_bytes() + fdas::tc2_template_bytes(M) : 0));
    *out = p;
    return FDAS_OK;
}

int fdas_plan_describe(fdas_plan p, fdas_plan_desc *d)
{
    if (!p || !d) return fail(FDAS_ERR_INVALID_ARG, "null argument");
    d->n_max = p->n_max;
    d->n_templates = p->M;
    d->tpl_len = p->K_user;
    d->frame_len = p->K;
    d->seg_len = p->L;
    d->seg_step = p->S;
    d->tpl_per_cta = p->g_auto ? 0 : p->G;
    d->precision = p->precision;
    d->device = p->device;
    d->device_bytes = p->device_bytes;
    d->tuned = p->tuned;
    for (int i = 0; i < 12; ++i) d->tune_ms[i] = p->tune_ms[i / 4][i % 4];
    d->tune_ms_tc = p->tune_ms_tc;
    d->batch_blocks = p->bk.resident;
    d->groups = p->ngroups;
    return FDAS_OK;
}

int fdas_plan_tpl_per_cta(fdas_plan p, int64_t n)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    if (n < 1 || n > p->n_max) return fail(FDAS_ERR_INVALID_ARG, "n=%lld outside [1, n_max=%lld]", (long long)n, (long long)p->n_max);
    return call_G(p, n_segments(p, n), p->M);
}

int fdas_convolve_batch(fdas_plan p, int count, const void *const *ins, const int64_t *ns, float *const *outs,
                        void *stream)
{
    int rc = validate_batch(p, count, ins, ns, outs);
    if (rc) return rc;
    if (count == 0) return FDAS_OK;
    std::lock_guard<std::mutex> lk(p->batch_mu);
    DeviceGuard g(p->device);
    if (!g.ok) return fail(FDAS_ERR_CUDA, "cannot select plan device %d", p->device);
    return enqueue_batch(p, count, ins, ns, outs, (cudaStream_t)stream);
}

int fdas_convolve(fdas_plan p, const void *in, int64_t n, float *out, void *stream)
{
    int rc = validate_convolve(p, in, n, out);
    if (rc) return rc;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(FDAS_ERR_CUDA, "cannot select plan device %d", p->device);
    CUtensorMap map;
    if ((rc = encode_input_map(&map, in, n))) return rc;
    if (p->d_rows) return launch_all(p, &map, base_args(p, n, out), n, (cudaStream_t)stream);
    return enqueue_segments(p, &map, n, out, 0, n_segments(p, n), (cudaStream_t)stream);
}

int fdas_convolve_direct(fdas_plan p, const void *in, int64_t n, float *out, void *stream)
{
    int rc = validate_convolve(p, in, n, out);
    if (rc) return rc;
    DeviceGuard g(p->device);
    if (!g.ok) return fail(FDAS_ERR_CUDA, "cannot select plan device %d", p->device);
    cudaError_t e = fdas::launch_td_direct(static_cast<const float2 *>(in), n, p->d_h32, p->M, p->K_user, out,
                                           (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "time-domain kernel launch");
    return FDAS_OK;
}

int fdas_convolve_candidates(fdas_plan p, const void *in, int64_t n, float threshold, fdas_candidate *cand,
                             int64_t max_cand, unsigned long long *count, void *stream)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    if (!in || !count || (max_cand > 0 && !cand)) return fail(FDAS_ERR_INVALID_ARG, "null pointer");
    if (max_cand < 0) return fail(FDAS_ERR_INVALID_ARG, "max_cand < 0");
    if (n < 1 || n > p->n_max) return fail(FDAS_ERR_INVALID_ARG, "n=%lld outside [1, n_max=%lld]", (long long)n, (long long)p->n_max);
    if (reinterpret_cast<uintptr_t>(in) % 16) return fail(FDAS_ERR_INVALID_ARG, "input pointer must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(count) % 8 || reinterpret_cast<uintptr_t>(cand) % 8)
        return fail(FDAS_ERR_INVALID_ARG, "counter and candidate array must be 8-byte aligned");
    if (p->precision == FDAS_PREC_TC_FP16)
        return fail(FDAS_ERR_UNSUPPORTED, "candidates are built for the FP32 and two-stage tensor-core forms");
    DeviceGuard g(p->device);
    if (!g.ok) return fail(FDAS_ERR_CUDA, "cannot select plan device %d", p->device);
    CUtensorMap map;
    int rc = encode_input_map(&map, in, n);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    FDAS_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned long long), s), "clear candidate counter");
    fdas::OlsArgs a = base_args(p, n, nullptr);
    a.cand = cand ? cand : reinterpret_cast<fdas_candidate *>(count);   // non-null selects the epilogue
    a.cand_count = count;
    a.cand_max = max_cand;
    a.threshold = threshold;
    if (p->precision == FDAS_PREC_TC_DFT2) {
        cudaError_t e = fdas::launch_ols_tc2(&map, a, p->d_H16, p->d_tc2c, p->eH, (int)n_segments(p, n), s);
        if (e != cudaSuccess) return cuda_fail(e, "segment kernel launch (two-stage tensor-core form, candidates)");
        return FDAS_OK;
    }
    return launch_all(p, &map, a, n, s);
}

int fdas_convolve_host(fdas_plan p, const void *in_host, int64_t n, float *out_host, void *stream)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    if (!in_host || !out_host) return fail(FDAS_ERR_INVALID_ARG, "null host pointer");
    if (n < 1 || n > p->n_max) return fail(FDAS_ERR_INVALID_ARG, "n=%lld outside [1, n_max=%lld]", (long long)n, (long long)p->n_max);
    std::lock_guard<std::mutex> lk(p->host_mu);
    DeviceGuard g(p->device);
    if (!g.ok) return fail(FDAS_ERR_CUDA, "cannot select plan device %d", p->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->d_in_stage) {
        FDAS_CUDA_TRY(cudaMalloc(&p->d_in_stage, sizeof(float2) * (size_t)p->n_max), "cudaMalloc input staging");
        FDAS_CUDA_TRY(cudaMalloc(&p->d_out_stage, sizeof(float) * (size_t)p->n_max * p->M), "cudaMalloc output staging");
        FDAS_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking), "copy stream");
        for (auto &ev : p->chunk_ev) FDAS_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
        p->device_bytes += (int64_t)(sizeof(float2) * (size_t)p->n_max + sizeof(float) * (size_t)p->n_max * p->M);
    }
    FDAS_CUDA_TRY(cudaMemcpyAsync(p->d_in_stage, in_host, sizeof(float2) * (size_t)n, cudaMemcpyHostToDevice, s), "H2D input");
    CUtensorMap map;
    int rc = encode_input_map(&map, p->d_in_stage, n);
    if (rc) return rc;
    if (p->d_rows) {   // grouped plans: every group writes every column range, one copy at the end
        if ((rc = launch_all(p, &map, base_args(p, n, p->d_out_stage), n, s))) return rc;
        FDAS_CUDA_TRY(cudaMemcpyAsync(out_host, p->d_out_stage, sizeof(float) * (size_t)n * p->M, cudaMemcpyDeviceToHost, s),
                      "D2H plane");
        FDAS_CUDA_TRY(cudaStreamSynchronize(s), "stream sync");
        return FDAS_OK;
    }
    const int64_t nseg = n_segments(p, n);
    const int chunks = (int)std::min<int64_t>(kMaxChunks, nseg);
    for (int c = 0; c < chunks; ++c) {
        const int64_t s0 = nseg * c / chunks, s1 = nseg * (c + 1) / chunks;
        if ((rc = enqueue_segments(p, &map, n, p->d_out_stage, s0, s1, s))) return rc;
        FDAS_CUDA_TRY(cudaEventRecord(p->chunk_ev[c], s), "event record");
        FDAS_CUDA_TRY(cudaStreamWaitEvent(p->copy_stream, p->chunk_ev[c], 0), "stream wait");
        const int64_t i0 = s0 * p->S, i1 = std::min<int64_t>(s1 * p->S, n);
        FDAS_CUDA_TRY(cudaMemcpy2DAsync(out_host + i0, sizeof(float) * n, p->d_out_stage + i0, sizeof(float) * n,
                                        sizeof(float) * (i1 - i0), p->M, cudaMemcpyDeviceToHost, p->copy_stream),
                      "D2H plane chunk");
    }
    FDAS_CUDA_TRY(cudaStreamSynchronize(p->copy_stream), "copy stream sync");
    FDAS_CUDA_TRY(cudaStreamSynchronize(s), "stream sync");
    return FDAS_OK;
}

int fdas_plan_status(fdas_plan p, void *stream)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    DeviceGuard g(p->device);
    FDAS_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
    int st = 0;
    FDAS_CUDA_TRY(cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
    if (st) {
        FDAS_CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(int)), "status clear");
        return fail(FDAS_ERR_TIMEOUT, "an in-kernel bounded wait ran out (status 0x%x)", st);
    }
    return FDAS_OK;
}

int fdas_destroy(fdas_plan p)
{
    if (!p) return fail(FDAS_ERR_INVALID_ARG, "null plan");
    plan_free(p);
    return FDAS_OK;
}

}  // extern "C"
