// morton.cuh -- Morton keys (Sec. 1.1 "Morton ordering"): the bits of the
// coordinates interleaved so that at every bit level the first coordinate is
// the most significant (key bit d*b + (d-1-j) is bit b of coordinate j).
// Shared by the encoder of the build and the point-by-point updater; it also
// compiles for the host.
#pragma once

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#ifndef __forceinline__
#define __forceinline__ inline
#endif
#endif

namespace zdk {
typedef unsigned long long u64;

// Spread the low 21 bits of x so that bit b lands on bit 3b.
__host__ __device__ __forceinline__ u64 spread3(u64 x)
{
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Spread the low 32 bits of x so that bit b lands on bit 2b.
__host__ __device__ __forceinline__ u64 spread2(u64 x)
{
    x &= 0xffffffffull;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

// Key bit d*b + (d-1-j) is bit b of coordinate j (x most significant).
template <int DIM>
__host__ __device__ __forceinline__ u64 interleave(u64 c0, u64 c1, u64 c2)
{
    if (DIM == 3) return (spread3(c0) << 2) | (spread3(c1) << 1) | spread3(c2);
    return (spread2(c0) << 1) | spread2(c1);
}

} // namespace zdk
