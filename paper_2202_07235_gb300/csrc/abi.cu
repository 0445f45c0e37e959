// Library-wide entry points: version, error strings, device status word,
// buffer-size queries.
#include <mutex>

#include "operand.cuh"
#include "ptx_sync.cuh"

namespace rsvd {

// One status word per device that loads the module (first failure wins;
// rsvd_status reads and clears it).
__device__ int g_status_word = 0;

RSVD_HIDDEN int* status_word() {
  static std::mutex mu;
  static int* ptrs[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
    ptrs[dev] = static_cast<int*>(p);
  }
  return ptrs[dev];
}

namespace {

// One thread waits on an mbarrier whose phase never completes (nothing
// arrives), with the bounded wait of the scoring kernels.
__global__ void wait_selftest_kernel(int* status, long long budget) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, budget)) record(status, kDevTimeout);
}

}  // namespace
}  // namespace rsvd

extern "C" {

int rsvd_selftest_wait_timeout(long long budget_cycles, void* stream) {
  if (budget_cycles < 1 || budget_cycles > (1LL << 31)) return RSVD_EINVAL;
  int* status = rsvd::status_word();
  if (!status) return RSVD_ECUDA;
  rsvd::wait_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(status, budget_cycles);
  return rsvd::launch_status();
}

int rsvd_abi_version(void) { return RSVD_ABI_VERSION; }

const char* rsvd_strerror(int code) {
  switch (code) {
    case RSVD_OK: return "ok";
    case RSVD_EINVAL: return "invalid argument (NULL pointer or inconsistent size)";
    case RSVD_EUNSUPPORTED: return "unsupported size or precision";
    case RSVD_ECUDA: return "CUDA runtime error";
    case RSVD_EDEVICE: return "device-side bounds check failed";
    case RSVD_ETIMEOUT: return "device-side wait timed out";
    case RSVD_EWORKSPACE: return "workspace missing or too small";
    case RSVD_ENOCONVERGE: return "eigen-solver did not converge";
    default: return "unknown status code";
  }
}

int rsvd_status(void* stream) {
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return RSVD_ECUDA;
  int* p = rsvd::status_word();
  if (!p) return RSVD_ECUDA;
  int v = 0;
  if (cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return RSVD_ECUDA;
  if (v != 0) {
    int zero = 0;
    if (cudaMemcpy(p, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return RSVD_ECUDA;
  }
  switch (v) {
    case rsvd::kDevOk: return RSVD_OK;
    case rsvd::kDevTimeout: return RSVD_ETIMEOUT;
    case rsvd::kDevNoConverge: return RSVD_ENOCONVERGE;
    default: return RSVD_EDEVICE;
  }
}

size_t rsvd_compressed_bytes(int N, int T, int H, int Q, int precision) {
  if (N <= 0 || T <= 0 || H <= 0 || Q <= 0) return 0;
  if (precision == RSVD_FP32) return (size_t)N * (size_t)T * (size_t)H * (size_t)(Q / 2) * 8u;
  rsvd::OperandLayout L{};
  if (!rsvd::is_operand_precision(precision) || !rsvd::make_operand_layout(N, T, H, Q, &L)) return 0;
  return rsvd::operand_bytes(L, precision);
}

}  // extern "C"
