// FP64 instantiation of the ENUF-DPD kernels and launch sequences.
#include "enuf_enqueue.cuh"
namespace enuf {
ENUF_INSTANTIATE(double)
}
