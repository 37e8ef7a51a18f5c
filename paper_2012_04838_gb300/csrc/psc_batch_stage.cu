// One RK stage of the persistent ensemble kernel (psc_batch_kernel.cuh),
// compiled once per stage (-DPSCB_STAGE=1..4) so the four build in parallel;
// psc_batch.cu launches them through the functions below.
#include "psc_batch_kernel.cuh"

#ifndef PSCB_STAGE
#error "define PSCB_STAGE"
#endif

#define PSCB_CAT(a, b) a##b
#define PSCB_NAME(a, b) PSCB_CAT(a, b)

cudaError_t PSCB_NAME(pscb_launch_stage_, PSCB_STAGE)(bool big, int grid, size_t smem, cudaStream_t st,
                                                       const void* head, const void* boxes, const void* segs,
                                                       void* counters) {
  auto k = big ? k_batch_stage<PSCB_STAGE, true> : k_batch_stage<PSCB_STAGE, false>;
  k<<<grid, kThreads, smem, st>>>(static_cast<const Head*>(head), static_cast<const PscBatchBox*>(boxes),
                                  static_cast<const Seg*>(segs), static_cast<unsigned char*>(counters));
  return cudaGetLastError();
}

// Allow `smem` bytes of dynamic shared memory and return the CTAs of this
// stage's kernel that fit on one SM at once.
int PSCB_NAME(pscb_prepare_stage_, PSCB_STAGE)(bool big, size_t smem) {
  auto k = big ? k_batch_stage<PSCB_STAGE, true> : k_batch_stage<PSCB_STAGE, false>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kThreads, smem);
  return per;
}
