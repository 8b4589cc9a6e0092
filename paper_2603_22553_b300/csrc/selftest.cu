// lpc_wait_selftest: a bounded device wait that completes or runs out on
// purpose, so that a host can check how the library reports a wait that runs
// out.  Every spin-wait of the step kernels (mbarrier waits on TMA copies,
// the grid barrier of the persistent batched launch) is bounded by a clock64
// budget; on expiry the kernel writes LPC_ERR_TIMEOUT to a status word and
// returns instead of hanging, and the host reads the word.  This kernel runs
// the same kind of bounded wait on a one-thread launch, with a budget the
// caller chooses, on an mbarrier or on a global flag that nothing completes.
#include "tma_ptx.cuh"

namespace lpc {
namespace {

constexpr long long kSelftestMaxCycles = 4000000000LL;   // the step kernels' bound (about 2 s)

// mode 0: mbarrier with no arrival; mode 1: flag that nothing sets;
// mode 2: mbarrier that completes before the wait (control)
__global__ void k_wait_selftest(int mode, long long budget, unsigned int* status,
                                const unsigned int* flag) {
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar, 1);
    fence_mbar_init();
    bool ok = true;
    if (mode == 1) {
        const long long t0 = clock64();
        while (*reinterpret_cast<const volatile unsigned int*>(flag) == 0u) {
            if (clock64() - t0 > budget) { ok = false; break; }
            __nanosleep(1000);
        }
    } else {
        if (mode == 2) mbar_arrive(&bar);
        if (!mbar_try_wait(&bar, 0u)) {
            const long long t0 = clock64();
            while (!mbar_try_wait(&bar, 0u))
                if (clock64() - t0 > budget) { ok = false; break; }
        }
    }
    *status = ok ? (unsigned int)LPC_OK : (unsigned int)LPC_ERR_TIMEOUT;
}

}  // namespace
}  // namespace lpc

using namespace lpc;

extern "C" lpc_status lpc_wait_selftest(int32_t mode, int64_t budget_cycles, void* stream) {
    if (mode < 0 || mode > 2) {
        set_error("lpc_wait_selftest: mode must be 0, 1 or 2");
        return LPC_ERR_INVALID;
    }
    if (budget_cycles < 1 || budget_cycles > kSelftestMaxCycles) {
        set_error("lpc_wait_selftest: budget_cycles must be in 1 .. 4e9");
        return LPC_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* words = nullptr;     // [0] status, [1] flag
    cudaError_t e = cudaMalloc(&words, 2 * sizeof(unsigned int));
    if (e != cudaSuccess) return cuda_fail(e, "lpc_wait_selftest: allocation");
    unsigned int host[2] = {0xffffffffu, 0u};
    e = cudaMemcpyAsync(words, host, sizeof host, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 1, 0, st>>>(mode, (long long)budget_cycles, words, words + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, words, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(words);
    if (e != cudaSuccess) return cuda_fail(e, "lpc_wait_selftest");
    if (host[0] == (unsigned int)LPC_ERR_TIMEOUT) {
        set_error("lpc_wait_selftest: the device wait ran out of its budget (kernel returned early)");
        return LPC_ERR_TIMEOUT;
    }
    if (host[0] != (unsigned int)LPC_OK) {
        set_error("lpc_wait_selftest: status word not written");
        return LPC_ERR_CUDA;
    }
    return LPC_OK;
}
