// The transcoding kernels with 128 compute threads of 48 input bytes each
// (6 KiB chunks), compiled for 3 resident CTAs per SM.
#define GBU_THREADS 128
#define GBU_BPT 48
#define GBU_MIN_BLOCKS 3
#define GBU_VNS v128x48
#define GBU_VARIANT_FN variant_128x48
#include "transcode.cuh"
