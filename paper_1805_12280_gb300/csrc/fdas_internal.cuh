// Internal declarations shared by the plan layer and the kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fdas.h"

namespace fdas {

// ---------------------------------------------------------------------------
// Segment FFT geometry.  L = 16 * Q * R points, NT = L / 16 threads, 16 values per
// thread.  Forward transform (decimation in frequency over the digits of n):
//   pass A  thread t = b*R + c holds x[a*NT + t], a < 16 -> 16-point DFT over a (k1),
//           twiddle W_L^{t k1};
//   pass B  thread holds (k1, c) groups, DFT over b (k2), twiddle W_{QR}^{c k2};
//   pass C  thread holds (k1, k2) groups, DFT over c (k3);
// X[k1 + 16 k2 + 16 Q k3] ends in registers ("C distribution").  The inverse runs
// the same passes backwards with conjugate twiddles and ends in natural order.
// ---------------------------------------------------------------------------
template <int L>
struct Geo {
    static_assert(L == 1024 || L == 2048 || L == 4096, "segment length");
    static constexpr int P = 16;
    static constexpr int Q = (L == 1024) ? 8 : 16;
    static constexpr int R = (L == 4096) ? 16 : 8;
    static constexpr int NT = L / 16;
    static constexpr int GB = 16 / Q;     // (k1, c) groups per thread in pass B
    static constexpr int GC = 16 / R;     // (k1, k2) groups per thread in pass C
    static constexpr int LD2 = NT + 1;    // padded row of the second exchange buffer
};

// Frequency index held in register slot j (0..15) of thread tau in the C distribution.
__host__ __device__ inline int freq_of_slot(int L, int tau, int j)
{
    const int Q = (L == 1024) ? 8 : 16;
    const int R = (L == 4096) ? 16 : 8;
    const int NT = L / 16;
    const int g = j / R, k3 = j % R;
    const int k1 = tau & 15;
    const int k2 = tau / 16 + (NT / 16) * g;
    return k1 + 16 * k2 + 16 * Q * k3;
}

// Arguments of the FP32 segment kernel.
struct OlsArgs {
    const float4 *H;      // [M][8][NT] float4 = two complex per thread slot pair
    const float2 *tw;     // [L] W_L^e = exp(-2 pi i e / L), FP32
    float *out;           // [M][n]
    int64_t n;
    int M, G, S, K;       // templates, templates per CTA, segment step, frame length
    int seg_begin;        // first segment of this launch
    int *status;          // device status word (bit 0: a bounded wait ran out)
    // candidate epilogue (fdas_convolve_candidates): crossings of `threshold`
    fdas_candidate *cand = nullptr;
    unsigned long long *cand_count = nullptr;
    long long cand_max = 0;
    float threshold = 0.f;
    // grouped plans: template z of this launch goes to plane row rows[z], its outputs shifted
    // by shifts[z] (the first nonzero tap); outputs before the shift are zero
    const int *rows = nullptr;
    const int *shifts = nullptr;
    // two-stage tensor-core form: fp16 template spectra, plan constants, their scale and the
    // template-pair groups per segment pair
    const unsigned char *H16 = nullptr;
    const unsigned char *cst = nullptr;
    int eH = 0, ng = 1;
};

// One array of a batch: its input tensor map (param space), output plane and work items.
struct BatchArray {   // aligned as CUtensorMap
    CUtensorMap map;      // 1-D tiled map over the array's complex64 input
    float *out;           // [M][n]
    int64_t n;
    int64_t item_off;     // index of the array's first work item
    int nseg;             // segments of this array
    int pad_;
};
constexpr int kBatchMax = 120;   // arrays per launch: the table is a kernel parameter (< 32 KB)
struct BatchTable {
    int count;
    int pad_;
    int64_t total_items;
    BatchArray arr[kBatchMax];
};
static_assert(sizeof(BatchTable) + sizeof(OlsArgs) + sizeof(int *) <= 32764, "batch table must fit the kernel parameters");

// Resolved persistent batch kernel for one segment length.
struct BatchKernel {
    const void *fn = nullptr;
    int block = 0;
    size_t smem = 0;
    int resident = 0;     // blocks that fit on the device at once
};
cudaError_t batch_kernel(int L, BatchKernel *k);

// A lane: one work counter, one host table and one graph [reset counter -> persistent
// kernel]; batches on different lanes may run concurrently.
struct Lane {
    int *d_counter = nullptr;
    BatchTable *table = nullptr;
    OlsArgs args = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t kernel_node = nullptr;
    int version = -1;
};
// Enqueue planes of `count` arrays (validated by the caller) on the lane, chunked by kBatchMax.
int lane_launch(fdas_plan p, Lane *l, int count, const void *const *ins, const int64_t *ns, float *const *outs,
                cudaStream_t stream);
void lane_free(Lane *l);
int validate_array(fdas_plan p, const void *in, int64_t n, const float *out);
int plan_templates(fdas_plan p);
int plan_grouped(fdas_plan p);
int plan_precision(fdas_plan p);      // FDAS_PREC_* of the plan
int *plan_status_word(fdas_plan p);   // the plan's device status word
int64_t plan_n_max(fdas_plan p);

// Graph-free launches of the persistent batch kernel with caller-provided work counters
// (one per table of kBatchMax arrays, at most max_chunks); clears them on the stream first.
int batch_direct(fdas_plan p, int count, const void *const *ins, const int64_t *ns, float *const *outs,
                 int *counters, int max_chunks, cudaStream_t stream);
int plan_device(fdas_plan p);
int set_error(int code, const char *msg);   // records the thread-local message, returns code

// Launch the FP32 segment kernel over segments [seg_begin, seg_begin + nseg); with a.cand
// set, the candidate epilogue replaces the plane stores.
cudaError_t launch_ols_fp32(int L, const CUtensorMap *tmap, const OlsArgs &a, int nseg,
                            cudaStream_t s);
size_t ols_fp32_smem_bytes(int L);

// Tensor-core form (L = 2048): the real DFT matrices (plan time) and the segment kernel.
cudaError_t launch_tc_matrices(unsigned char *wmat, cudaStream_t s);
size_t tc_matrix_bytes();
cudaError_t launch_ols_tc(const CUtensorMap *tmap, const OlsArgs &a, const unsigned char *wmat, int nseg,
                          cudaStream_t s);

// Two-stage tensor-core form (L = 2048): plan constants (the two real DFT matrices and the
// twiddle table), the fp16 template spectra, and the segment kernel over segments
// [a.seg_begin, a.seg_begin + nseg).
size_t tc2_const_bytes();
size_t tc2_template_bytes(int M);
cudaError_t launch_tc2_constants(unsigned char *cst, cudaStream_t s);
cudaError_t launch_tc2_pretransform(const float2 *h32, int M, int K, const double2 *w64, int eH, unsigned char *H16,
                                    cudaStream_t s);
cudaError_t launch_ols_tc2(const CUtensorMap *tmap, const OlsArgs &a, const unsigned char *H16,
                           const unsigned char *cst, int eH, int nseg, cudaStream_t s);
// Its persistent batch kernel (same parameters as the FP32 one) and the template-pair groups
// per segment pair for a launch over n_sp segment pairs.
cudaError_t tc2_batch_kernel(BatchKernel *k);
int tc2_groups_for(int64_t n_sp, int M);

// Time-domain form (Eq. 1 term by term) over the raw templates h [M][K].
cudaError_t launch_td_direct(const float2 *x, int64_t n, const float2 *h, int M, int K, float *out, cudaStream_t s);

// Plan-time kernels (FP64).
cudaError_t launch_twiddles(int L, double2 *w64, float2 *w32, cudaStream_t s);
// Full-length FD-FIR passes (P = 2048 * P2): forward transform of in[0, len) into A (times
// scale); inverse of X . H into the power row out[0, n) through the scratch B.
cudaError_t fdfir_forward(int P2, const float2 *in, int64_t len, const float2 *tw1, const float2 *tw2, float2 *A,
                          float scale, cudaStream_t s);
cudaError_t fdfir_inverse(int P2, const float2 *X, const float2 *H, float2 *B, const float2 *tw1, const float2 *tw2,
                          float *out, int64_t n, cudaStream_t s);
// split: the slot pairs (c, 8 + c) as (re_c, re_{8+c}, im_c, im_{8+c}) (tensor-core form),
// else the slot pairs (2p, 2p + 1) as two complex values.
cudaError_t launch_pretransform(int L, const float2 *h32, int M, int K, const double2 *w64,
                                float4 *Hperm, bool split, cudaStream_t s);

}  // namespace fdas
