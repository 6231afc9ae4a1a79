// The transcoding kernels with 512 compute threads of 48 input bytes each
// (24 KiB chunks), compiled for 1 resident CTA per SM.
#define GBU_THREADS 512
#define GBU_BPT 48
#define GBU_MIN_BLOCKS 1
#define GBU_VNS v512x48
#define GBU_VARIANT_FN variant_512x48
#include "transcode.cuh"
