// Device helpers: D3Q19 constants, population storage formats, Philox4x32-10.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "lbt_internal.h"

namespace lbt {

// D3Q19 velocity set: rest, +-x, +-y, +-z, then the 12 edge vectors in
// opposite pairs.  Indices are compile-time after unrolling, so these fold
// into immediates.
__host__ __device__ constexpr int cvec(int i, int a)
{
    constexpr int c[kQ][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                              {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                              {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                              {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return c[i][a];
}

template <class T>
__host__ __device__ constexpr T wgt(int i)
{
    return i == 0 ? T(1) / T(3) : (i < 7 ? T(1) / T(18) : T(1) / T(36));
}

// ---- storage formats -------------------------------------------------------
// Every format stores the deviation d_i = f_i - w_i.  E: stored element type,
// A: arithmetic type, R: type of boundary samples and of field read-outs.
template <int ST>
struct Stor;

template <>
struct Stor<kF64> {
    using E = double;
    using A = double;
    using R = double;
    static __device__ __forceinline__ A in(E v) { return v; }
    static __device__ __forceinline__ E out(A v) { return v; }
};

template <>
struct Stor<kF32> {
    using E = float;
    using A = float;
    using R = float;
    static __device__ __forceinline__ A in(E v) { return v; }
    static __device__ __forceinline__ E out(A v) { return v; }
};

template <>
struct Stor<kF16> {
    using E = uint16_t;
    using A = float;
    using R = float;
    static __device__ __forceinline__ A in(E v) { return __half2float(__ushort_as_half(v)); }
    static __device__ __forceinline__ E out(A v) { return __half_as_ushort(__float2half_rn(v)); }
};

template <>
struct Stor<kBF16> {
    using E = uint16_t;
    using A = float;
    using R = float;
    static __device__ __forceinline__ A in(E v) { return __bfloat162float(__ushort_as_bfloat16(v)); }
    static __device__ __forceinline__ E out(A v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
};

// A vector of VW consecutive stored elements moved with one load/store.
template <int BYTES>
struct RawOf;
template <>
struct RawOf<16> {
    using T = uint4;
};
template <>
struct RawOf<8> {
    using T = uint2;
};
template <>
struct RawOf<4> {
    using T = unsigned int;
};
template <>
struct RawOf<2> {
    using T = unsigned short;
};

template <class E, int VW>
struct Pack {
    using Raw = typename RawOf<sizeof(E) * VW>::T;
    union {
        Raw raw;
        E e[VW];
    };
};

template <class Raw>
__device__ __forceinline__ Raw ld_nc(const Raw* p)
{
    return __ldg(p);
}
template <>
__device__ __forceinline__ unsigned short ld_nc<unsigned short>(const unsigned short* p)
{
    return __ldg(p);
}

template <class Raw>
__device__ __forceinline__ Raw zero_raw()
{
    Raw r;
    memset(&r, 0, sizeof(Raw));
    return r;
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ----------------------
// 32-bit words throughout: the 32x32 multiplies run at the full integer rate,
// while 64x64 products (a 64-bit variant) go through a much slower path.
__device__ __forceinline__ void philox4x32_10(uint32_t x[4], uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t hi0 = __umulhi(M0, x[0]), lo0 = M0 * x[0];
        const uint32_t hi1 = __umulhi(M1, x[2]), lo1 = M1 * x[2];
        const uint32_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
        x[0] = y0;
        x[1] = lo1;
        x[2] = y2;
        x[3] = lo0;
    }
}

// Unit-variance uniform number on [-sqrt3, sqrt3) from a 32-bit word in the
// precision of the bead dynamics: FP64 from all 32 bits (u = v 2^-32, exact),
// FP32 from the top 24 bits (exact uniform grid, scaled by sqrt 3).
template <class T>
__device__ __forceinline__ T unit_uniform_t(uint32_t v);
template <>
__device__ __forceinline__ double unit_uniform_t<double>(uint32_t v)
{
    const double u01 = (double)v * (1.0 / 4294967296.0);  // 2^-32
    return sqrt(3.0) * (2.0 * u01 - 1.0);
}
template <>
__device__ __forceinline__ float unit_uniform_t<float>(uint32_t v)
{
    const float u01 = (float)(v >> 8) * (1.0f / 16777216.0f);  // 2^-24
    return 1.7320508075688772f * (2.0f * u01 - 1.0f);
}

// Reciprocal of the bead pair forces: correctly rounded division in FP64,
// the hardware's approximate reciprocal in FP32 (PTX rcp.approx.ftz.f32, at
// most one ulp off, far below the FP32 dynamics' own rounding; the pair
// arguments are never subnormal).  One instruction: the MD substeps are a
// latency-bound chain, and the approximate division intrinsic it replaces
// cost half of a substep's force phase.
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int wrapi(int v, int E) { return v < 0 ? v + E : (v >= E ? v - E : v); }

// Time-interpolation weights of the four ring samples j-1, j, j+1, j+2 for
// the boundary velocity at t = n + 1, t in (jK, (j+1)K].
template <class R>
struct TimeWeights {
    int slot[4];
    R c[4];
};

template <class R>
__device__ __forceinline__ TimeWeights<R> time_weights(int64_t n, int K, int mode, int ring_slots)
{
    TimeWeights<R> tw;
    // 32-bit division while the step fits (a 64-bit one is a long instruction sequence)
    const int64_t j = n < 0x7fffffff ? (int64_t)((uint32_t)n / (uint32_t)K) : n / K;
    int s = (int)(n + 1 - j * K);
    R th = (R)s / (R)K;
    for (int a = 0; a < 4; a++) {
        const int64_t jj = j - 1 + a;
        tw.slot[a] = jj < 0x7fffffff ? (int)(((int)jj % ring_slots + ring_slots) % ring_slots)
                                     : (int)(((jj % ring_slots) + ring_slots) % ring_slots);
        tw.c[a] = R(0);
    }
    if (mode == 0) {
        tw.c[1] = R(1) - th;
        tw.c[2] = th;
    } else {
        R h00 = 2 * th * th * th - 3 * th * th + 1;
        R h10 = th * th * th - 2 * th * th + th;
        R h01 = -2 * th * th * th + 3 * th * th;
        R h11 = th * th * th - th * th;
        if (j >= 1) {
            tw.c[0] = -R(0.5) * h10;
            tw.c[1] = h00 - R(0.5) * h11;
            tw.c[2] = h01 + R(0.5) * h10;
            tw.c[3] = R(0.5) * h11;
        } else {
            tw.c[1] = h00 - h10 - R(0.5) * h11;
            tw.c[2] = h01 + h10;
            tw.c[3] = R(0.5) * h11;
        }
    }
    return tw;
}

// Substep s = n + 1 - jK (1 .. K) of the step n -> n + 1 within its coarse interval j.
__device__ __forceinline__ int mlp_substep(int64_t n, int K)
{
    const int64_t j = n < 0x7fffffff ? (int64_t)((uint32_t)n / (uint32_t)K) : n / K;
    return (int)(n + 1 - j * K);
}

// Learned residual of the boundary velocity (upsampler boxes): output row of
// the face site, substep s.  Loaded before the time interpolation of the ring
// samples (the two loads overlap), added after it.
__device__ __forceinline__ void load_mlp_residual(const SCParams& p, const BoxDev& bd, int s, int f, int pp, int qq,
                                                  float r[3])
{
    if (bd.mlp_row < 0) return;
    const float* y = p.mlp_y + (int64_t)(3 * (s - 1)) * p.mlp_ystride + bd.mlp_row + ((int64_t)f * bd.E + qq) * bd.E + pp;
    for (int c = 0; c < 3; c++) r[c] = y[c * p.mlp_ystride];
}
template <class R>
__device__ __forceinline__ void add_mlp_residual(const SCParams& p, const BoxDev& bd, const float r[3], R ub[3])
{
    if (bd.mlp_row < 0) return;
    for (int c = 0; c < 3; c++) ub[c] += (R)(p.mlp_yunit * r[c]);
}

// Owning face of a boundary site (first velocity face containing it in the
// order x-, x+, y-, y+, z-, z+) and its in-face coordinates.
__device__ __forceinline__ int owning_face(int x, int y, int z, int E, int per, int& p, int& q)
{
    if (!(per & 1) && x == 0) { p = y; q = z; return 0; }
    if (!(per & 1) && x == E - 1) { p = y; q = z; return 1; }
    if (!(per & 2) && y == 0) { p = x; q = z; return 2; }
    if (!(per & 2) && y == E - 1) { p = x; q = z; return 3; }
    if (!(per & 4) && z == 0) { p = x; q = y; return 4; }
    p = x; q = y;
    return 5;
}

// Time-interpolated velocity at coarse face point (P, Q) from the ring.
template <class R>
__device__ __forceinline__ void coarse_velocity(const R* ring, int64_t slot_elems, int64_t ring_off, int Ec, int f,
                                                int P, int Q, const TimeWeights<R>& tw, R u[3])
{
    const int64_t fe = (int64_t)Ec * Ec;
    const int64_t site = (int64_t)Q * Ec + P;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        R acc = R(0);
        for (int a = 0; a < 4; a++) {
            if (tw.c[a] != R(0)) {  // a zero weight never touches its (possibly unpushed) slot
                const R* base = ring + (int64_t)tw.slot[a] * slot_elems + ring_off;
                acc += tw.c[a] * base[((int64_t)f * 3 + c) * fe + site];
            }
        }
        u[c] = acc;
    }
}

// Boundary velocity of face site (p, q): the ring holds every sample on the
// face sites (a zoomed box's coarse samples are interpolated bilinearly onto
// them when pushed, see bilinear_face_site), so a step interpolates in time
// only (Sec. 3: bilinear in space, interpolated in time).
template <class R>
__device__ __forceinline__ void boundary_velocity(const R* ring, int64_t slot_elems, const BoxDev& bd, int f, int p,
                                                  int q, const TimeWeights<R>& tw, R u[3])
{
    coarse_velocity<R>(ring, slot_elems, bd.ring_off, bd.E, f, p, q, tw, u);
}

// Component c of face f of a coarse sample [6][3][Ec][Ec] (point P at site
// P z) at face site (p, q): bilinear interpolation between the four coarse
// points around it, the last point standing in past the grid's end.
template <class R>
__host__ __device__ inline R bilinear_face_site(const R* coarse, int Ec, int z, int f, int c, int p, int q)
{
    const int P0 = p / z, Q0 = q / z;
    const int P1 = P0 + 1 < Ec ? P0 + 1 : P0, Q1 = Q0 + 1 < Ec ? Q0 + 1 : Q0;
    const R fp = (R)(p - P0 * z) / (R)z, fq = (R)(q - Q0 * z) / (R)z;
    const R* g = coarse + ((int64_t)f * 3 + c) * Ec * Ec;
    const R u00 = g[(int64_t)Q0 * Ec + P0], u10 = g[(int64_t)Q0 * Ec + P1];
    const R u01 = g[(int64_t)Q1 * Ec + P0], u11 = g[(int64_t)Q1 * Ec + P1];
    return (R(1) - fq) * ((R(1) - fp) * u00 + fp * u10) + fq * ((R(1) - fp) * u01 + fp * u11);
}

}  // namespace lbt
