// Failure detection without a fault: a kernel whose only mbarrier nothing
// ever arrives at.  Its bounded wait (the one every tensor-core kernel here
// uses) gives up after the given limit, records CDMD_ERR_TIMEOUT in the
// context's status word and returns, so the context stays usable.
#include "tc_common.cuh"

namespace cdmd {
namespace {

__global__ void __launch_bounds__(32) selftest_wait_kernel(uint64_t limit_ns, int* status) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) tc::mbar_wait(&bar, 0u, &abort_flag, status, limit_ns);
    __syncwarp();
}

// r[i] = rcp64(a[i]), q[i] = rsqrt64(a[i]): the small solves' reciprocal and
// reciprocal square root, exposed so that a test can bound their error.
__global__ void selftest_recip_kernel(const double* __restrict__ a, int64_t n, double* __restrict__ r,
                                      double* __restrict__ q) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = a[i];
    if (r) r[i] = rcp64(x);
    if (q) q[i] = rsqrt64(x);
}

}  // namespace

cdmd_status launch_selftest_recip(const double* a, int64_t n, double* r, double* q, cudaStream_t stream) {
    if (n == 0) return CDMD_OK;
    selftest_recip_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(a, n, r, q);
    CDMD_CHECK_LAUNCH("selftest_recip_kernel");
    return CDMD_OK;
}

cdmd_status launch_selftest_wait(cdmd_ctx* ctx, uint64_t limit_ns, cudaStream_t stream) {
    selftest_wait_kernel<<<1, 32, 0, stream>>>(limit_ns, ctx->d_status);
    CDMD_CHECK_LAUNCH("selftest_wait_kernel");
    return CDMD_OK;
}

}  // namespace cdmd
