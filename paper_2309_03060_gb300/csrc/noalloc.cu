// Allocation-free Kronecker MVM.
//
// The regular entry points draw their intermediate buffers from a context's
// workspace, which grows with cudaMalloc.  Some callers cannot let a library
// allocate device memory at all: code that owns every byte of the device
// through its own memory pool, code that runs where an allocation would
// implicitly synchronise the device, and callers that never create a
// context.  cola_kron_matvec_noalloc serves them: it computes the same FP32
// Kronecker MVM as cola_matvec with COLA_PREC_F32 (the cyclic mode products
// of the SIMT GEMM), but its intermediate results live in one file-scope
// device array of fixed size, g_kron_scratch, that every GPU loading this
// library holds until the process exits.
#include <mutex>

#include "internal.h"

namespace {

// 2 x 4 Mi floats = 32 MiB: two ping-pong halves for the intermediate mode
// products.
constexpr int64_t kScratchHalf = (int64_t)4 << 20;
static __device__ __align__(256) float g_kron_scratch[2 * kScratchHalf];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_addr[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};

}  // namespace

using namespace cola;

extern "C" cola_status cola_kron_matvec_noalloc(int nfactors, const int64_t* rows,
                                                const int64_t* cols, const float* const* factors,
                                                const float* X, float* Y, int64_t nrhs,
                                                cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(nfactors >= 1 && nfactors <= 8, COLA_ERR_INVALID_ARG, "nfactors = %d",
                 nfactors);
    COLA_REQUIRE(rows && cols && factors && X && Y, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(nrhs >= 1, COLA_ERR_INVALID_ARG, "nrhs = %lld", (long long)nrhs);
    COLA_REQUIRE(X != Y, COLA_ERR_INVALID_ARG, "X and Y must not alias");
    // Every size below is checked before it is formed, so no product can wrap
    // around and slip past the scratch bound.
    constexpr int64_t kMax = INT64_MAX;
    int64_t cur = 1, maxsz = 0;
    for (int k = 0; k < nfactors; ++k) {
      COLA_REQUIRE(rows[k] >= 1 && cols[k] >= 1 && factors[k], COLA_ERR_INVALID_ARG,
                   "factor %d: bad shape or NULL data", k);
      COLA_REQUIRE(cur <= kMax / cols[k], COLA_ERR_INVALID_ARG,
                   "the product of the factor column counts overflows int64");
      cur *= cols[k];
    }
    // intermediate sizes of the cyclic steps (all but the last go to scratch)
    for (int k = 0; k + 1 < nfactors; ++k) {
      const int64_t rest = cur / cols[k];
      COLA_REQUIRE(rest <= kMax / rows[k], COLA_ERR_INVALID_ARG,
                   "intermediate %d of the mode products overflows int64", k);
      cur = rest * rows[k];
      maxsz = std::max(maxsz, cur);
    }
    COLA_REQUIRE(maxsz == 0 || nrhs <= kScratchHalf / maxsz, COLA_ERR_INVALID_ARG,
                 "nrhs = %lld times the largest intermediate (%lld floats) exceeds the fixed "
                 "scratch of %lld floats per half",
                 (long long)nrhs, (long long)maxsz, (long long)kScratchHalf);

    int dev = 0;
    COLA_CUDA(cudaGetDevice(&dev));
    COLA_REQUIRE(dev >= 0 && dev < kMaxDevices, COLA_ERR_UNSUPPORTED, "device %d", dev);
    float* scratch;
    {
      // set-up, once per device, with that device current
      std::lock_guard<std::mutex> lock(g_setup_mutex);
      if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        COLA_CUDA(cudaGetSymbolAddress(&ptr, g_kron_scratch));
        COLA_CUDA(cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev));
        g_scratch_addr[dev] = (float*)ptr;
      }
      scratch = g_scratch_addr[dev];
    }

    // A context-free launcher state on the stack: no workspace is touched.
    Ctx c;
    c.device = dev;
    c.num_sms = g_num_sms[dev];
    c.s = (cudaStream_t)stream;
    int64_t size = 1;
    for (int k = 0; k < nfactors; ++k) size *= cols[k];
    const float* in = X;
    for (int k = 0; k < nfactors; ++k) {
      const int64_t n_in = cols[k], n_out = rows[k];
      const int64_t rest = size / n_in, out_size = rest * n_out;
      const bool last = (k == nfactors - 1);
      float* out = last ? Y : scratch + (k & 1) * kScratchHalf;
      // D[rest, i] = sum_j X[j, rest] K[i, j]   (factor row-major, packed)
      gemm<float>(&c, rest, n_out, n_in, 1.0, in, 1, rest, size, factors[k], 1, n_in, 0, 0.0,
                  out, n_out, 1, out_size, nrhs);
      in = out;
      size = out_size;
    }
  });
}
