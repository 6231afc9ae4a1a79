// The transcoding kernels with 256 compute threads of 32 input bytes each
// (8 KiB chunks), compiled for 2 resident CTAs per SM.
#define GBU_THREADS 256
#define GBU_BPT 32
#define GBU_MIN_BLOCKS 2
#define GBU_VNS v256x32
#define GBU_VARIANT_FN variant_256x32
#include "transcode.cuh"
