// Fluctuating lattice Boltzmann collision (the thermal fluid of the hybrid
// method the paper builds on, Sec. 1: Ahlrichs-Duenweg coupling of beads to a
// fluctuating lattice Boltzmann fluid, so that kT > 0 is consistent on the
// fluid side as well as on the beads).
//
// The collision acts on the moments of the D3Q19 orthogonal basis: 19 integer
// polynomials e_k(c) of the lattice velocity with
//     sum_i w_i e_k(c_i) e_l(c_i) = b_k delta_kl.
// Modes 0 .. 3 (mass, momentum) are conserved.  Mode k >= 4 of the
// non-equilibrium part f - f^eq is multiplied by gamma_k and receives noise of
// the variance the fluctuation-dissipation theorem fixes,
//     m_k* = gamma_k m_k^neq + sqrt(mu rho b_k (1 - gamma_k^2)) xi_k,
//     mu = kT / c_s^2,
// and the populations come back as f_i* = f_i^eq + w_i sum_k e_k(c_i) m_k* / b_k.
// gamma_k = 1 - 1/tau for every k and kT = 0 is the BGK collision.
//
// Noise: Philox4x32-10 (Salmon et al., SC'11), counter (step, site, block,
// 0xF1) for blocks 0 .. 3, key = the box's seed; words 0 .. 14 in block order
// go to modes 4 .. 18, each mapped to a unit-variance uniform on
// [-sqrt 3, sqrt 3) (all 32 bits in FP64, the top 24 in FP32).
#pragma once
#include "lbt_device.cuh"

namespace lbt {

// e_k(c_i): the orthogonal D3Q19 polynomials, k = 0 .. 18.
__host__ __device__ constexpr int emode(int k, int i)
{
    const int x = cvec(i, 0), y = cvec(i, 1), z = cvec(i, 2);
    const int c2 = x * x + y * y + z * z;
    switch (k) {
        case 0: return 1;
        case 1: return x;
        case 2: return y;
        case 3: return z;
        case 4: return c2 - 1;
        case 5: return 3 * x * x - c2;
        case 6: return y * y - z * z;
        case 7: return x * y;
        case 8: return y * z;
        case 9: return z * x;
        case 10: return (3 * c2 - 5) * x;
        case 11: return (3 * c2 - 5) * y;
        case 12: return (3 * c2 - 5) * z;
        case 13: return (y * y - z * z) * x;
        case 14: return (z * z - x * x) * y;
        case 15: return (x * x - y * y) * z;
        case 16: return 3 * c2 * c2 - 6 * c2 + 1;
        case 17: return (2 * c2 - 3) * (3 * x * x - c2);
        default: return (2 * c2 - 3) * (y * y - z * z);
    }
}

// b_k = sum_i w_i e_k(c_i)^2, as a multiple of 1/36 (w_i 36 is 12, 2 or 1).
__host__ __device__ constexpr int bnorm36(int k)
{
    int s = 0;
    for (int i = 0; i < kQ; i++) s += (i == 0 ? 12 : (i < 7 ? 2 : 1)) * emode(k, i) * emode(k, i);
    return s;
}

// Deviation of the equilibrium of population i: f_i^eq - w_i =
// w_i (drho + rho (3 cu + 4.5 cu^2 - usq)), usq = 1.5 u^2.
template <class A>
__device__ __forceinline__ A fluct_deq(int i, A drho, A rho, A ux, A uy, A uz, A usq)
{
    A cu = A(0);
    if (cvec(i, 0)) cu += cvec(i, 0) * ux;
    if (cvec(i, 1)) cu += cvec(i, 1) * uy;
    if (cvec(i, 2)) cu += cvec(i, 2) * uz;
    return wgt<A>(i) * (drho + rho * (A(3) * cu + A(4.5) * cu * cu - usq));
}

// Fluctuating collision of one site (global index `site` within its box) at
// step n from its pulled deviations d_i = f_i - w_i (overwritten) with moments
// drho = sum d and u = j / rho; writes the post-collision deviations to out.
// fd: relaxation factors, noise amplitudes and seed of the box.  The noise of
// modes 4 + 4 blk .. 7 + 4 blk comes from Philox block blk, drawn as the modes
// are formed.
template <class A>
__device__ __forceinline__ void fluct_collide(A d[kQ], A drho, A ux, A uy, A uz, const FluctDev& fd, int64_t n,
                                              int site, A out[kQ])
{
    const uint64_t seed = fd.seed;
    const A rho = A(1) + drho;
    const A usq = A(1.5) * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < kQ; i++) d[i] -= fluct_deq<A>(i, drho, rho, ux, uy, uz, usq);  // f_i - f_i^eq
    const A srho = sqrt(rho);
    A mk[15];  // relaxed non-equilibrium moments plus noise, over b_k
#pragma unroll
    for (int blk = 0; blk < 4; blk++) {
        uint32_t x[4] = {(uint32_t)n, (uint32_t)site, (uint32_t)blk, 0xF1u};
        philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
        for (int w = 0; w < 4; w++) {
            const int k = 4 + 4 * blk + w;
            if (k < kQ) {
                A m = A(0);
#pragma unroll
                for (int i = 0; i < kQ; i++) {
                    const int e = emode(k, i);
                    if (e == 1) m += d[i];
                    else if (e == -1) m -= d[i];
                    else if (e != 0) m += A(e) * d[i];
                }
                // gamma and amplitude are the same for the whole warp: broadcast loads
                const A g = (A)fd.gamma[k - 4], am = (A)fd.amp[k - 4];
                mk[k - 4] = (g * m + am * srho * unit_uniform_t<A>(x[w])) * (A(36) / A(bnorm36(k)));
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        A s = A(0);
#pragma unroll
        for (int k = 4; k < kQ; k++) {
            const int e = emode(k, i);
            if (e == 1) s += mk[k - 4];
            else if (e == -1) s -= mk[k - 4];
            else if (e != 0) s += A(e) * mk[k - 4];
        }
        out[i] = fluct_deq<A>(i, drho, rho, ux, uy, uz, usq) + wgt<A>(i) * s;
    }
}

}  // namespace lbt
