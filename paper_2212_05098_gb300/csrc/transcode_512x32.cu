// The transcoding kernels with 512 compute threads of 32 input bytes each
// (16 KiB chunks), compiled for 1 resident CTA per SM.
#define GBU_THREADS 512
#define GBU_BPT 32
#define GBU_MIN_BLOCKS 1
#define GBU_VNS v512x32
#define GBU_VARIANT_FN variant_512x32
#include "transcode.cuh"
