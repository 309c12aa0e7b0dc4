// Host stand-in for the few CUDA runtime types named in the library's
// internal declarations, so that its layout helpers compile with g++ for the
// CPU checks under tests/host_emu (nothing here is called).
#pragma once
typedef int cudaError_t;
typedef struct CUstream_st* cudaStream_t;
struct int2 { int x, y; };
