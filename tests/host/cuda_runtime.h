// Host stand-in for the CUDA runtime header, for the warp emulation of the
// finder (tests only): the few types the library's internal header names.
#pragma once
#include <cstdint>
typedef void *cudaStream_t;
typedef int cudaError_t;
enum { cudaSuccess = 0 };
inline int cudaGetDevice(int *d) { *d = 0; return 0; }
inline int cudaSetDevice(int) { return 0; }
struct float4 { float x, y, z, w; };
struct float2 { float x, y; };
inline float2 make_float2(float x, float y) { return float2{x, y}; }
inline float4 make_float4(float x, float y, float z, float w) { return float4{x, y, z, w}; }
