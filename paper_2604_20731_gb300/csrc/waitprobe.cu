// A kernel that runs the bounded-wait protocol of this library's kernels on
// demand, so that a test can watch a device-side wait expire without any
// fault: it waits on an mbarrier that nobody completes (or, with `arrive`,
// one that a second thread completes) while it holds tensor memory and has a
// bulk copy of its own in flight.  On expiry it does what every kernel here
// does: it records bit 8 in its status word, waits (bounded) for its own copy
// to land, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace adsgb {
namespace {

__global__ void __launch_bounds__(32) k_wait_probe(const void* src, unsigned long long limit_ns, int arrive,
                                                   int* word) {
  __shared__ __align__(16) unsigned char buf[16];
  __shared__ __align__(8) uint64_t mb_copy, mb_wait;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init_cta(&mb_copy, 1);
    mbar_init_cta(&mb_wait, 1);
    mbar_arrive_tx(&mb_copy, sizeof(buf));
    bulk_load(buf, src, sizeof(buf), &mb_copy);
  }
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tbase)),
               "r"(32));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tbase;
  if (arrive && tid == 1) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&mb_wait)) : "memory");
  const bool ok = mbar_wait_for(&mb_wait, 0, limit_ns);
  if (!ok && tid == 0) atomicOr(word, 8);
  mbar_wait_for(&mb_copy, 0, limit_ns);  // the copy in flight lands before the CTA's memory goes
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncwarp();
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32));
}

}  // namespace

cudaError_t launch_wait_probe(const void* src16, unsigned long long limit_ns, int arrive, int* word,
                              cudaStream_t st) {
  if (!src16 || (reinterpret_cast<uintptr_t>(src16) & 15) || !word) return cudaErrorInvalidValue;
  k_wait_probe<<<1, 32, 0, st>>>(src16, limit_ns, arrive, word);
  return cudaGetLastError();
}

}  // namespace adsgb
