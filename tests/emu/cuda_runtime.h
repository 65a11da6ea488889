// Host stand-ins for the CUDA names that eri_device.cuh and the generated ERI
// kernels use, so that tests/test_kernel_emulation.py can compile the
// generated kernel code as plain C++ and run it one thread at a time on the
// CPU (test infrastructure: the library itself never runs this way).
// Placed first on the include path, this file replaces <cuda_runtime.h>.
#pragma once
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __launch_bounds__(...)
#define __restrict__
#define __constant__

struct int2 { int x, y; };
struct int4 { int x, y, z, w; };
struct float2 { float x, y; };
struct float4 { float x, y, z, w; };
struct double2 { double x, y; };
struct double4 { double x, y, z, w; };
struct emu_dim3 { unsigned x, y, z; };
extern emu_dim3 blockIdx, threadIdx, blockDim, gridDim;
typedef void* cudaStream_t;

using std::fma;
using std::fmax;
using std::fabs;
using std::sqrt;
inline int min(int a, int b) { return a < b ? a : b; }
inline long long min(long long a, long long b) { return a < b ? a : b; }
inline int max(int a, int b) { return a > b ? a : b; }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
inline float fmaf(float a, float b, float c) { return std::fma(a, b, c); }
template <class T> inline T __ldg(const T* p) { return *p; }
inline double atomicAdd(double* p, double v) { const double o = *p; *p = o + v; return o; }
inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
    const unsigned long long o = *p; *p = o + v; return o;
}
inline unsigned long long atomicMax(unsigned long long* p, unsigned long long v) {
    const unsigned long long o = *p; if (v > o) *p = v; return o;
}
inline unsigned int atomicMax(unsigned int* p, unsigned int v) { const unsigned int o = *p; if (v > o) *p = v; return o; }
inline float __fdividef(float a, float b) { return a / b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fdiv_rn(float a, float b) { return a / b; }
inline int __double2int_rn(double x) { return (int)std::nearbyint(x); }
inline int __float2int_rn(float x) { return (int)std::nearbyint(x); }
inline long long __double_as_longlong(double x) { long long r; std::memcpy(&r, &x, 8); return r; }
inline double __longlong_as_double(long long x) { double r; std::memcpy(&r, &x, 8); return r; }
inline unsigned int __float_as_uint(float x) { unsigned int r; std::memcpy(&r, &x, 4); return r; }
inline double __dadd_rn(double a, double b) { return a + b; }
// one thread at a time: a warp of one lane, whose shuffles return its own value
#define GB_WARP_SIZE 1
template <class T> inline T __shfl_down_sync(unsigned, T v, int) { return v; }
template <class T> inline T __shfl_up_sync(unsigned, T v, int) { return v; }
template <class T> inline T __shfl_xor_sync(unsigned, T v, int) { return v; }
inline double __dsub_rn(double a, double b) { return a - b; }
