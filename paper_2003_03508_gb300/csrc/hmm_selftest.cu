// Check of the library's failure detection on the device: the bounded wait
// that every tensor-core kernel uses on its mbarriers (hmm_tc_common.cuh)
// must give up, flag ETIMEOUT in the status word and return, rather than hang,
// when the phase it waits for never completes. The kernel waits on a fresh
// mbarrier whose phase nothing completes, with a short limit; nothing faults,
// traps or spins without bound.
#include "hmm_tc_common.cuh"

namespace hmm {
namespace {

__global__ void wait_selftest_kernel(long long limit_cycles, unsigned *status, long long *waited) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);  // one arrival completes phase 0; none is made
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        const bool ok = mbar_wait(&bar, 0, &abort_flag, status, limit_cycles);
        *waited = clock64() - t0;
        if (ok) atomicOr(status, ST_EINVAL);  // the phase cannot have completed
    }
}

}  // namespace
}  // namespace hmm

using namespace hmm;

extern "C" int hmm_check_bounded_wait(int device, double limit_ms, double *waited_ms) {
    if (!(limit_ms > 0.0) || limit_ms > 2000.0) return HMM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return HMM_ECUDA;
    int khz = 0;
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device) != cudaSuccess || khz <= 0) return HMM_ECUDA;
    const long long limit = (long long)(limit_ms * (double)khz);  // cycles at the rated clock
    unsigned *d_status = nullptr;
    long long *d_waited = nullptr;
    cudaError_t e = cudaMalloc(&d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&d_waited, sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32>>>(limit, d_status, d_waited);
        e = cudaGetLastError();
    }
    unsigned st = 0;
    long long cyc = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&cyc, d_waited, sizeof(long long), cudaMemcpyDeviceToHost);
    if (d_status) cudaFree(d_status);
    if (d_waited) cudaFree(d_waited);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HMM_ECUDA;
    }
    if (waited_ms) *waited_ms = (double)cyc / (double)khz;
    if (st & ST_EINVAL) return HMM_EINVAL;
    return (st & ST_ETIMEOUT) ? HMM_ETIMEOUT : HMM_OK;
}
