// The transcoding kernels with 256 compute threads of 48 input bytes each
// (12 KiB chunks), compiled for 2 resident CTAs per SM.
#define GBU_THREADS 256
#define GBU_BPT 48
#define GBU_MIN_BLOCKS 2
#define GBU_VNS v256x48
#define GBU_VARIANT_FN variant_256x48
#include "transcode.cuh"
