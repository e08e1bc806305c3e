// Primitives of the Gray-code walk shared by the enumeration kernels.
//
// Reflected Gray code over the IB inner spins: step t (1 .. 2^IB - 1)
// flips spin ctz(t) to the value of that bit in gray(t) = t ^ (t >> 1).  The 16-bit
// view of an int32 energy or field is floor(x / 2^16); two walks share one
// 32-bit register as the integer hi * 2^16 + lo, so one 32-bit add advances
// both exactly while every lane stays inside [0, 2^16).
#pragma once

#include "bf_internal.cuh"

namespace bf {

__host__ __device__ constexpr int cx_ctz(int t) { return (t & 1) ? 0 : 1 + cx_ctz(t >> 1); }
// value (1 = +1) of the spin flipped by step t of the reflected Gray code
__host__ __device__ constexpr bool cx_up(int t) { return (((t ^ (t >> 1)) >> cx_ctz(t)) & 1) != 0; }

// integer packing hi * 2^16 + lo of the 16-bit views of two int32 values
__device__ __forceinline__ unsigned pack_hi16(int lo, int hi)
{
    return ((unsigned)(hi >> 16) << 16) + (unsigned)(lo >> 16);
}

// 16-bit views of two energies, biased by 2^31 so that both lanes are non-negative
__device__ __forceinline__ unsigned pack_energy(int lo, int hi)
{
    return (((unsigned)hi + 0x80000000u) & 0xffff0000u) | (((unsigned)lo + 0x80000000u) >> 16);
}

// 16-bit threshold that catches every exact energy <= tau (see the bound in k_gray.cu)
__device__ __forceinline__ unsigned threshold16(int tau)
{
    unsigned th = (((unsigned)tau + 0x80000000u) >> 16) + 1u;
    return th > 0xffffu ? 0xffffu : th;
}

template <int IB>
struct Packed {
    unsigned Xa, Xb, M;
    unsigned Ga[IB], Gb[IB];
};

}  // namespace bf
