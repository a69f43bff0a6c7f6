// Plain FP64 form of the solver.
#include "sim_impl.cuh"

namespace pncg {
Sim *make_sim_f64() { return new SimImpl<double>(); }

// Failure-detection self-test: one block arrives at a counter that expects two arrivals and waits on it with the
// grid barriers' bounded wait; nothing completes it, so the wait gives up after limit_ns and sets ERR_TIMEOUT.
static __global__ void k_wait_selftest(unsigned int *count, uint32_t *err, unsigned long long limit_ns)
{
    if (threadIdx.x != 0) return;
    red_release_add(count, 1u);
    wait_count(count, 2u, err, limit_ns);
}

sim_status wait_selftest(double limit_s, std::string &msg)
{
    if (!(limit_s > 0.0 && limit_s <= 4.0)) { msg = "limit_s must be in (0, 4]"; return SIM_ERR_INVALID_ARG; }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        msg = "no CUDA device";
        return SIM_ERR_CUDA;
    }
    unsigned int *buf = nullptr;   // [0] the arrival counter, [1] the error word
    cudaError_t e = cudaMalloc(&buf, 2 * sizeof(unsigned int));
    if (e != cudaSuccess) { msg = cudaGetErrorString(e); return SIM_ERR_CUDA; }
    e = cudaMemset(buf, 0, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>(buf, buf + 1, (unsigned long long)(limit_s * 1e9));
        e = cudaGetLastError();
    }
    unsigned int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, buf + 1, sizeof err, cudaMemcpyDeviceToHost);   // waits for the kernel
    cudaFree(buf);
    if (e != cudaSuccess) { msg = cudaGetErrorString(e); return SIM_ERR_CUDA; }
    if (err & ERR_TIMEOUT) { msg = "device wait timed out (the self-test's expected outcome)"; return SIM_ERR_TIMEOUT; }
    msg = "the self-test's wait completed";
    return SIM_OK;
}
}
