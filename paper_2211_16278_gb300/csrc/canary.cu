// Workspace canaries (debug option BBLOCK_OPT_CHECKS): every field, converted-input block
// and partial block the library places in its workspace is followed by kCanaryBytes of a
// fixed pattern, written before a wave's kernels run and verified after its reduction. A
// kernel that wrote past the end of its block changes a canary, which sets kStatusCanary in
// the context's status word (reported by bblock_status). No access is made outside the
// workspace: the canaries are part of it.
#include "bblock_internal.h"

namespace bb {
namespace {

constexpr uint32_t kCanaryWord = 0xA5C3A5C3u;

__global__ void k_canaries(uint32_t* const* __restrict__ list, int n, int check,
                           int* __restrict__ status) {
  constexpr int kWords = kCanaryBytes / 4;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    uint32_t* c = list[i];
    for (int w = threadIdx.x; w < kWords; w += blockDim.x) {
      if (!check) {
        c[w] = kCanaryWord;
      } else if (c[w] != kCanaryWord) {
        atomicOr(status, kStatusCanary);
      }
    }
  }
}

}  // namespace

cudaError_t launch_canaries(uint32_t* const* d_list, int n, bool check, int* status,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int grid = n < 4096 ? n : 4096;
  k_canaries<<<grid, 64, 0, s>>>(d_list, n, check ? 1 : 0, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bb
