// FP32 instantiation of the ENUF-DPD kernels and launch sequences.
#include "enuf_enqueue.cuh"
namespace enuf {
ENUF_INSTANTIATE(float)
// the batched launch sequence runs FP32 systems
template size_t batch_bytes<float>(const BatchSys*, int);
template cudaError_t batch_build<float>(void*, const BatchSys*, int, BatchLaunch*);
template cudaError_t batch_enqueue<float>(const BatchLaunch&, cudaStream_t, cudaStream_t, cudaEvent_t, cudaEvent_t,
                                          LaunchLog*);
}
