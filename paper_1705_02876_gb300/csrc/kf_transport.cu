// Batched covariance transport C <- J C J^T for general dense 6x6 J: the
// many-small-matrices product the paper benchmarks on the GPU (Section 4.1:
// 6x6 products in a Matriplex-style layout against batched cuBLAS), here one
// thread per matrix with J and C in registers.  The fit's own transport
// exploits J's structure (kf_math.cuh); this kernel assumes none.
#include "kf.h"
#include "kf_api_internal.h"

namespace kf {
namespace {

// J [36][n] row-major per matrix, C [21][n] packed lower triangle (in place).
// A = J C one row at a time; row i of the result is A[i][:] J^T, of which the
// lower triangle (k <= i) is stored.
__global__ void __launch_bounds__(256) transport_batch_kernel(int64_t n, const float *__restrict__ Jg,
                                                              float *__restrict__ Cg)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        float J[36], C[21];
#pragma unroll
        for (int i = 0; i < 36; ++i) J[i] = __ldcs(Jg + i * n + t);
#pragma unroll
        for (int i = 0; i < 21; ++i) C[i] = __ldcs(Cg + i * n + t);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            float A[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                float acc = 0.0f;
#pragma unroll
                for (int m = 0; m < 6; ++m) acc = fmaf(J[i * 6 + m], C[pk(m, k)], acc);
                A[k] = acc;
            }
#pragma unroll
            for (int k = 0; k <= i; ++k) {
                float acc = 0.0f;
#pragma unroll
                for (int m = 0; m < 6; ++m) acc = fmaf(A[m], J[k * 6 + m], acc);
                __stcs(Cg + pk(i, k) * n + t, acc);
            }
        }
    }
}

}  // namespace
}  // namespace kf

using namespace kf;

extern "C" int kf_transport_batch(kf_context *ctx, int64_t n, const float *J, float *C, kf_stream stream_)
{
    if (!ctx) return KF_ERR_ARG;
    if (n < 0) return set_error(ctx, KF_ERR_ARG, "n must be >= 0");
    if (n == 0) return KF_OK;
    int rc;
    if ((rc = check_ptr(ctx, J, 4, "J")) || (rc = check_ptr(ctx, C, 4, "C"))) return rc;
    DeviceGuard dg(context_device(ctx));
    const int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)context_sm_count(ctx) * 8 * 4;
    transport_batch_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, reinterpret_cast<cudaStream_t>(stream_)>>>(
        n, J, C);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KF_OK : cuda_error(ctx, e, "transport launch");
}
