// Stream-collide with the boundary layer, staged through shared memory by
// TMA bulk copies (cp.async.bulk) in a warp-specialised pipeline.
//
// A tile is kSites consecutive sites of one box.  For population i the sites
// of a tile pull from one contiguous source range shifted by c_iy E + c_iz E^2
// (and by c_ix inside the row), so one bulk copy per population, widened by a
// 16-byte halo on each side for the x shift, brings everything the tile needs
// into shared memory; the x shift becomes an offset into that row.
//
// One producer warp claims tiles from a global counter and issues their 19
// copies into a ring of stages; a "full" barrier per stage counts the bytes
// landing, an "empty" barrier counts the consumer warps done with the stage.
// Fifteen consumer warps take the stages in order.  A consumer warp loads its
// sites' populations from the stage into registers and releases the stage at
// once, then collides and stores straight to global memory, so the copies of
// a later tile into that stage overlap the arithmetic and the stores of this
// one.  No block-wide barrier is taken inside the loop.
//
// Only sites whose pull source crosses a periodic face (a wrap) read global
// memory directly.  Copies are clamped to the box's arrays; sites whose
// source lies outside are boundary sites, which are overwritten with the
// boundary equilibrium anyway.
#pragma once
#include "lbt_device.cuh"
#include "lbt_fluct.cuh"

namespace lbt {

constexpr int kStagedHaloBytes = 16;  // x-shift halo on each side of a row
constexpr int kStagedConsumerWarps = 15;  // + the producer: four warps per scheduler
constexpr int kStagedConsumers = kStagedConsumerWarps * 32;
constexpr int kStagedThreads = kStagedConsumers + 32;  // + the producer warp
constexpr int kStagedHeaderBytes = 4096;               // barriers and tile headers
constexpr int kStagedMaxStages = 6;

// Tile geometry for SPT sites per consumer thread.  As many stages as fit in
// the 227 KB of shared memory a block may use (at most six).
template <int ST, int SPT>
struct Staged {
    using E = typename Stor<ST>::E;
    static constexpr int kSites = kStagedConsumers * SPT;
    static constexpr int kRowBytes = kSites * (int)sizeof(E);               // one population row of a tile
    static constexpr int kRowStride = kRowBytes + 2 * kStagedHaloBytes;
    static constexpr int kStageBytes = kQ * kRowStride;
    static constexpr int kFit = (227 * 1024 - kStagedHeaderBytes) / kStageBytes;
    static constexpr int kStages = kFit > kStagedMaxStages ? kStagedMaxStages : kFit;
    static constexpr int kSmemBytes = kStagedHeaderBytes + kStages * kStageBytes;
    static constexpr int kHalo = kStagedHaloBytes / (int)sizeof(E);         // halo elements
    static_assert(kStages >= 2, "tile too large for a two-stage pipeline");
    static_assert(kRowStride % 16 == 0, "bulk copies need 16-byte aligned rows");
};

// Sites per consumer thread the staged kernel supports per storage format
// (the first is the default): FP64 1; FP32 2 or 1; 16-bit 2 or 1.
inline bool staged_spt_ok(int storage, int spt) { return spt == 1 || (spt == 2 && storage != kF64); }
inline int staged_default_spt(int storage) { return storage == kF64 ? 1 : 2; }
inline int staged_tile_sites(int spt) { return kStagedConsumers * spt; }

// ---- PTX helpers (mbarrier + bulk copy) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// The populations stream through L2 once per step (both buffers together
// exceed it): their stores, and with chains in the launch (SCParams::
// hint_loads) also the bulk copies of the pulled rows, go in with the
// evict-first policy, so that what is reused -- the boundary sample ring, box
// records, the bead kernel's code and data -- stays in L2.  (Measured: the
// evict-first loads make the chain-free 256^3 sweep slower, the 128^3 step
// with its bead kernel faster.)
constexpr bool kL2HintStores = true;

__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Store of one population value or pair, evict-first when the hints are on.
template <class T>
__device__ __forceinline__ void st_stream(T* p, T v)
{
    if constexpr (kL2HintStores) __stcs(p, v);
    else *p = v;
}

// Test the phase; a thread that finds it incomplete may be suspended in
// hardware for up to 20 us (or until the phase completes) instead of spinning
// and taking issue slots from the warps that compute.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase), "r"(20000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for a phase of the barrier, giving up after limit_ns nanoseconds (one
// second by default; shorter only when a test makes a wait run out on purpose).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, int64_t limit_ns)
{
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, phase))
        if (global_ns() - t0 > (uint64_t)limit_ns) return false;
    return true;
}

// Box of tile t (the largest b with tile_prefix[b] <= t), searched by a whole
// warp: 32 candidates per round, so 512 boxes take two dependent loads.
__device__ __forceinline__ int locate_box_warp(const SCParams& p, int64_t t, int lane)
{
    int lo = 0, hi = p.nboxes - 1;
    while (lo < hi) {
        const int step = (hi - lo + 32) / 32;
        const int idx = lo + lane * step;
        const bool le = idx <= hi && p.tile_prefix[idx] <= t;
        const unsigned m = __ballot_sync(0xffffffffu, le);  // a prefix of the lanes; lane 0 always (prefix[lo] <= t)
        lo += (31 - __clz(m)) * step;
        hi = min(hi, lo + step - 1);
    }
    return lo;
}

// Shared-memory header: full and empty barriers, then the tile header the
// producer writes for each stage before it arms the barrier: the box record,
// first site, frozen flag, and what the collision and the boundary layer of
// the box need at this step -- BGK constants in the arithmetic type, the ring
// slots and weights of the time interpolation, the upsampler substep -- so
// that they are worked out (64-bit divisions, FP64 conversions, global loads)
// once per tile by the producer, not once per consumer warp.
template <int ST>
struct StagedTile {
    using A = typename Stor<ST>::A;
    using R = typename Stor<ST>::R;
    BoxDev bd;
    int64_t s0;
    int32_t box;
    int32_t mlp_s;
    int32_t frozen;  // the box carries an error status: its state does not change
    int32_t slot[4];
    R c[4];
    A om, om1, srcfac, drho_b;  // 1/tau, 1 - 1/tau, 1 - 1/(2 tau), rho_b - 1
};
// Consumers keep reading a tile's header after they have released its data
// stage (early release), so headers live in a ring of twice the stages: tile
// k uses header k mod 2S, which the producer rewrites for tile k + 2S only
// after every consumer warp has released tile k + S -- that is, after each of
// them has finished tile k (a warp takes the tiles in order).
template <int ST>
struct StagedHeader {
    uint64_t full[kStagedMaxStages];
    uint64_t empty[kStagedMaxStages];
    StagedTile<ST> t[2 * kStagedMaxStages];
};
static_assert(sizeof(StagedHeader<kF64>) <= kStagedHeaderBytes, "header does not fit");
static_assert(sizeof(StagedHeader<kF32>) <= kStagedHeaderBytes, "header does not fit");

// Quotient and remainder of a site index by E with a precomputed multiplier:
// q = (s * m) >> 40 with m = ceil(2^40 / E), exact for s < 2^31 and E <= 1024.
__device__ __forceinline__ int div_e(int64_t s, uint64_t m) { return (int)(((uint64_t)s * m) >> 40); }

// Consumer thread c (0 .. 479) of one tile: sites s0 + c + k 480, so the lanes
// of a warp read consecutive shared-memory words and store consecutive global
// words.  Populations go to registers, the warp releases the stage, then the
// collision (BGK with the equilibrium of opposite pairs shared: the even part
// in c.u is common, the odd part changes sign) and the stores.
template <int ST, int SPT, bool PER, bool ACCEL>
__device__ __forceinline__ void staged_tile(const SCParams& p, const StagedTile<ST>& th, const unsigned char* stage,
                                            uint64_t* empty)
{
    using S = Stor<ST>;
    using E = typename S::E;
    using A = typename S::A;
    using R = typename S::R;
    constexpr int H = Staged<ST, SPT>::kHalo;
    constexpr int C = kStagedConsumers;
    const int tid = threadIdx.x;
    // site indices of a box fit 32 bits (E <= 1024)
    const int s0 = (int)th.s0;
    const BoxDev& bd = th.bd;

    const int Ei = bd.E;
    const int n3 = (int)bd.n3;
    // body acceleration of the step in the arithmetic type, converted once
    A acA[3] = {A(0), A(0), A(0)};
    if (ACCEL)
        for (int c = 0; c < 3; c++) acA[c] = (A)bd.accel[c];
    const uint64_t mE = bd.div_magic;
    const int per = bd.per_mask;
    const bool px = per & 1, py = per & 2, pz = per & 4;
    const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
    E* Bb = reinterpret_cast<E*>(p.B) + bd.f_off;

    // coordinates of site k (recomputed where needed rather than held in
    // registers across the population loads)
    auto coords = [&](int k, int& x, int& y, int& z) {
        const int s = s0 + tid + k * C;
        const int sc = s < n3 ? s : 0;
        const int row = div_e(sc, mE);
        x = sc - row * Ei;
        z = div_e(row, mE);
        y = row - z * Ei;
    };
    int xs_[SPT], ys_[SPT], zs_[SPT];
    bool act[SPT], bnd[SPT];
    bool any_bnd = false;
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        act[k] = s0 + tid + k * C < n3;
        int x, y, z;
        coords(k, x, y, z);
        xs_[k] = x;
        ys_[k] = y;
        zs_[k] = z;
        bnd[k] = act[k] && ((!px && (x == 0 || x == Ei - 1)) || (!py && (y == 0 || y == Ei - 1)) ||
                            (!pz && (z == 0 || z == Ei - 1)));
        any_bnd |= bnd[k];
    }

    // f_i pulled into site k: shared memory, or global memory across a periodic
    // wrap; zero where it is not used (boundary and inactive sites)
    A f[kQ][SPT];
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        const int cx = cvec(i, 0), cy = cvec(i, 1), cz = cvec(i, 2);
        const E* row = reinterpret_cast<const E*>(stage + i * Staged<ST, SPT>::kRowStride);
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            A v = S::in(row[H + tid + k * C - cx]);
            if (PER) {
                const int xs = xs_[k] - cx, ys = ys_[k] - cy, zs = zs_[k] - cz;
                const bool wrap = (px && (xs < 0 || xs >= Ei)) || (py && (ys < 0 || ys >= Ei)) ||
                                  (pz && (zs < 0 || zs >= Ei));
                if (wrap && act[k])
                    v = S::in(Ab[(int64_t)i * n3 + ((int64_t)wrapi(zs, Ei) * Ei + wrapi(ys, Ei)) * Ei + wrapi(xs, Ei)]);
            }
            f[i][k] = (act[k] && !bnd[k]) ? v : A(0);
        }
    }
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(empty);  // this warp is done with the stage

    A drho[SPT], ux[SPT], uy[SPT], uz[SPT];
    bool nonfinite = false;  // a density that is not finite or not positive
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        A r = A(0), jx = A(0), jy = A(0), jz = A(0);
#pragma unroll
        for (int i = 0; i < kQ; i++) {
            r += f[i][k];
            if (cvec(i, 0)) jx += cvec(i, 0) * f[i][k];
            if (cvec(i, 1)) jy += cvec(i, 1) * f[i][k];
            if (cvec(i, 2)) jz += cvec(i, 2) * f[i][k];
        }
        const A rho = A(1) + r;
        nonfinite |= !(rho > A(0) && rho < A(1e30));  // NaN fails both comparisons
        const A inv = A(1) / rho;
        if (ACCEL) {
            jx += A(0.5) * rho * acA[0];
            jy += A(0.5) * rho * acA[1];
            jz += A(0.5) * rho * acA[2];
        }
        drho[k] = r;
        ux[k] = jx * inv;
        uy[k] = jy * inv;
        uz[k] = jz * inv;
    }
    // flag the box (it freezes from the next step on); boundary and inactive
    // sites pulled zeros, so only collided sites can raise the flag
    if (__any_sync(0xffffffffu, nonfinite) && (tid & 31) == 0) atomicCAS(&p.status[th.box], 0, LB_ERR_NONFINITE);
    // boundary sites: equilibrium of the boundary velocity from the ring
    if (any_bnd) {
        TimeWeights<R> tw;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            tw.slot[a] = th.slot[a];
            tw.c[a] = th.c[a];
        }
        const R* ring = reinterpret_cast<const R*>(p.ring);
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            if (bnd[k]) {
                int pp, qq, x, y, z;
                if (PER) {
                    x = xs_[k];
                    y = ys_[k];
                    z = zs_[k];
                } else {
                    coords(k, x, y, z);
                }
                const int fc = owning_face(x, y, z, Ei, per, pp, qq);
                float res[3];
                load_mlp_residual(p, bd, th.mlp_s, fc, pp, qq, res);
                R ub[3];
                boundary_velocity<R>(ring, p.ring_slot_elems, bd, fc, pp, qq, tw, ub);
                add_mlp_residual<R>(p, bd, res, ub);
                drho[k] = th.drho_b;
                ux[k] = (A)ub[0];
                uy[k] = (A)ub[1];
                uz[k] = (A)ub[2];
            }
        }
    }
    const A om = th.om, om1 = th.om1, srcfac = th.srcfac;
    A usq[SPT], rho_[SPT], ua[SPT];
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        usq[k] = A(1.5) * (ux[k] * ux[k] + uy[k] * uy[k] + uz[k] * uz[k]);
        rho_[k] = A(1) + drho[k];
        if (ACCEL) ua[k] = ux[k] * acA[0] + uy[k] * acA[1] + uz[k] * acA[2];
    }
    // post-collision value of population i at site k from its equilibrium deviation
    // populations are written in order 0, 1, ..., 18 through one running
    // pointer (row of population i at this thread's first site)
    E* out = Bb + s0 + tid;
    auto emit = [&](int i, int k, A deq, A cu) {
        A val = deq;
        if (!bnd[k]) {
            val = om1 * f[i][k] + om * deq;
            if (ACCEL) {
                const A w = wgt<A>(i);
                A ca = A(0);  // c_i . a in the arithmetic type (FP64 is slow on this part)
                if (cvec(i, 0)) ca += cvec(i, 0) * acA[0];
                if (cvec(i, 1)) ca += cvec(i, 1) * acA[1];
                if (cvec(i, 2)) ca += cvec(i, 2) * acA[2];
                val += srcfac * w * rho_[k] * (A(3) * (ca - ua[k]) + A(9) * cu * ca);
            }
        }
        // population 0 and odd i at `out`, the even partner of a pair one row further
        const int row = (i > 0 && (i & 1) == 0) ? n3 : 0;
        if (act[k]) st_stream(out + row + k * C, S::out(val));
    };
#pragma unroll
    for (int k = 0; k < SPT; k++) emit(0, k, wgt<A>(0) * (drho[k] - rho_[k] * usq[k]), A(0));
    // opposite pairs (1,2), (3,4), ..., (17,18)
#pragma unroll
    for (int i = 1; i < kQ; i += 2) {
        out += i == 1 ? n3 : 2 * n3;  // row of population i; population i + 1 is one row further
        const A w = wgt<A>(i);
        const int cx = cvec(i, 0), cy = cvec(i, 1), cz = cvec(i, 2);
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            A cu = A(0);
            if (cx) cu += cx * ux[k];
            if (cy) cu += cy * uy[k];
            if (cz) cu += cz * uz[k];
            const A even = w * (drho[k] + rho_[k] * (A(4.5) * cu * cu - usq[k]));
            const A odd = (A(3) * w) * rho_[k] * cu;
            emit(i, k, even + odd, cu);
            emit(i + 1, k, even - odd, -cu);
        }
    }
}

// ---- two adjacent sites per consumer thread (FP32 and 16-bit storage) -----
// Packed FP32 arithmetic: one instruction advances both sites of a thread.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one packed FMA: b (-1) is exact, so this is a - b rounded once
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Loads and stores of a pair of adjacent stored elements: one aligned word
// for the pair of a thread (elements e, e + 1 with e even), two scalar loads
// for the x-shifted pairs, conversions to and from FP32 packed where the
// format has a packed instruction (round to nearest even, as Stor<ST>::out).
template <int ST>
struct PairIO;
template <>
struct PairIO<kF32> {
    using E = float;
    static __device__ __forceinline__ float2 even(const E* row, int e) { return *reinterpret_cast<const float2*>(row + e); }
    static __device__ __forceinline__ float2 any(const E* row, int e) { return make_float2(row[e], row[e + 1]); }
    static __device__ __forceinline__ void store(E* p, float2 v) { st_stream(reinterpret_cast<float2*>(p), v); }
};
template <>
struct PairIO<kF16> {
    using E = uint16_t;
    static __device__ __forceinline__ float2 even(const E* row, int e)
    {
        return __half22float2(*reinterpret_cast<const __half2*>(row + e));
    }
    static __device__ __forceinline__ float2 any(const E* row, int e)
    {
        return make_float2(__half2float(__ushort_as_half(row[e])), __half2float(__ushort_as_half(row[e + 1])));
    }
    static __device__ __forceinline__ void store(E* p, float2 v)
    {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        st_stream(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<const unsigned int*>(&h));
    }
};
template <>
struct PairIO<kBF16> {
    using E = uint16_t;
    static __device__ __forceinline__ float2 even(const E* row, int e)
    {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(row + e));
    }
    static __device__ __forceinline__ float2 any(const E* row, int e)
    {
        return make_float2(__bfloat162float(__ushort_as_bfloat16(row[e])),
                           __bfloat162float(__ushort_as_bfloat16(row[e + 1])));
    }
    static __device__ __forceinline__ void store(E* p, float2 v)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        st_stream(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<const unsigned int*>(&h));
    }
};

// Consumer thread c (0 .. 479) of one tile of 960 sites takes the adjacent
// sites s0 + 2c and s0 + 2c + 1 (same row: E and s0 are even), so a warp
// reads and writes 64 consecutive sites with one word per lane.  Same
// arithmetic as staged_tile, on both sites at once; a boundary site takes
// om = 1, 1 - om = 0 and no force term in its lane, which turns the
// collision into its equilibrium.
template <int ST, bool PER, bool ACCEL>
__device__ __forceinline__ void staged_tile_pair(const SCParams& p, const StagedTile<ST>& th, const unsigned char* stage,
                                                 uint64_t* empty)
{
    static_assert(ST != kF64, "the paired body works in FP32");
    using S = Stor<ST>;
    using E = typename S::E;
    using IO = PairIO<ST>;
    constexpr int H = Staged<ST, 2>::kHalo;
    const int tid = threadIdx.x;
    const int s0 = (int)th.s0;
    const BoxDev& bd = th.bd;
    const int Ei = bd.E;
    const int n3 = (int)bd.n3;
    const int per = bd.per_mask;
    const bool px = per & 1, py = per & 2, pz = per & 4;
    const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
    E* Bb = reinterpret_cast<E*>(p.B) + bd.f_off;

    const int s = s0 + 2 * tid;  // first site of the pair (even)
    const bool act = s < n3;     // n3 is even: both sites or none
    int x, y, z;
    {
        const int sc = act ? s : 0;
        const int row = div_e(sc, bd.div_magic);
        x = sc - row * Ei;
        z = div_e(row, bd.div_magic);
        y = row - z * Ei;
    }
    const bool brow = (!py && (y == 0 || y == Ei - 1)) || (!pz && (z == 0 || z == Ei - 1));
    const bool bnd0 = act && (brow || (!px && x == 0));
    const bool bnd1 = act && (brow || (!px && x + 1 == Ei - 1));
    const bool keep0 = act && !bnd0, keep1 = act && !bnd1;

    // f_i pulled into both sites (zero where unused)
    float2 f[kQ];
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        const int cx = cvec(i, 0), cy = cvec(i, 1), cz = cvec(i, 2);
        const E* row = reinterpret_cast<const E*>(stage + i * Staged<ST, 2>::kRowStride);
        float2 v = cx == 0 ? IO::even(row, H + 2 * tid) : IO::any(row, H + 2 * tid - cx);
        if (PER) {
            const int ys = y - cy, zs = z - cz;
            const bool wyz = (py && (ys < 0 || ys >= Ei)) || (pz && (zs < 0 || zs >= Ei));
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const int xs = x + k - cx;
                const bool wrap = wyz || (px && (xs < 0 || xs >= Ei));
                if (wrap && act) {
                    const float w = S::in(
                        Ab[(int64_t)i * n3 + ((int64_t)wrapi(zs, Ei) * Ei + wrapi(ys, Ei)) * Ei + wrapi(xs, Ei)]);
                    if (k == 0) v.x = w;
                    else v.y = w;
                }
            }
        }
        // boundary lanes keep what they pulled (finite: the stage holds copied
        // or zeroed elements only); it is multiplied by zero below
        f[i] = v;
    }
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(empty);  // this warp is done with the stage

    // moments (sum of deviations, momentum)
    float2 r = f[0];
#pragma unroll
    for (int i = 1; i < kQ; i++) r = add2(r, f[i]);
    float2 jx = sub2(f[1], f[2]), jy = sub2(f[3], f[4]), jz = sub2(f[5], f[6]);
    jx = add2(jx, sub2(f[7], f[8]));
    jy = add2(jy, sub2(f[7], f[8]));
    jx = add2(jx, sub2(f[9], f[10]));
    jy = sub2(jy, sub2(f[9], f[10]));
    jx = add2(jx, sub2(f[11], f[12]));
    jz = add2(jz, sub2(f[11], f[12]));
    jx = add2(jx, sub2(f[13], f[14]));
    jz = sub2(jz, sub2(f[13], f[14]));
    jy = add2(jy, sub2(f[15], f[16]));
    jz = add2(jz, sub2(f[15], f[16]));
    jy = add2(jy, sub2(f[17], f[18]));
    jz = sub2(jz, sub2(f[17], f[18]));
    float2 rho = add2(f2(1.f), r);
    const bool nonfinite = (keep0 && !(rho.x > 0.f && rho.x < 1e30f)) || (keep1 && !(rho.y > 0.f && rho.y < 1e30f));
    if (__any_sync(0xffffffffu, nonfinite) && (tid & 31) == 0) atomicCAS(&p.status[th.box], 0, LB_ERR_NONFINITE);
    float2 ac[3] = {f2(0.f), f2(0.f), f2(0.f)};
    if (ACCEL) {
        for (int c = 0; c < 3; c++) ac[c] = f2((float)bd.accel[c]);
        const float2 hr = mul2(f2(0.5f), rho);
        jx = fma2(hr, ac[0], jx);
        jy = fma2(hr, ac[1], jy);
        jz = fma2(hr, ac[2], jz);
    }
    // 1 / rho by the fast reciprocal (within 2 ulp; the FP32 collision rounds
    // O(1) terms at 2^-24 anyway)
    const float2 inv = make_float2(__fdividef(1.f, rho.x), __fdividef(1.f, rho.y));
    float2 ux = mul2(jx, inv), uy = mul2(jy, inv), uz = mul2(jz, inv);
    float2 drho = r;

    // boundary sites: equilibrium of the boundary velocity from the ring
    if (bnd0 || bnd1) {
        TimeWeights<float> tw;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            tw.slot[a] = th.slot[a];
            tw.c[a] = th.c[a];
        }
        const float* ring = reinterpret_cast<const float*>(p.ring);
#pragma unroll 1
        for (int k = 0; k < 2; k++) {  // one lane at a time: fewer live registers
            if (k == 0 ? bnd0 : bnd1) {
                int pp, qq;
                const int fc = owning_face(x + k, y, z, Ei, per, pp, qq);
                float res[3];
                load_mlp_residual(p, bd, th.mlp_s, fc, pp, qq, res);
                float ub[3];
                boundary_velocity<float>(ring, p.ring_slot_elems, bd, fc, pp, qq, tw, ub);
                add_mlp_residual<float>(p, bd, res, ub);
                if (k == 0) {
                    drho.x = th.drho_b;
                    ux.x = ub[0];
                    uy.x = ub[1];
                    uz.x = ub[2];
                } else {
                    drho.y = th.drho_b;
                    ux.y = ub[0];
                    uy.y = ub[1];
                    uz.y = ub[2];
                }
            }
        }
        rho = add2(f2(1.f), drho);
    }

    // per-lane relaxation: boundary lanes take their equilibrium
    const float2 om = make_float2(bnd0 ? 1.f : th.om, bnd1 ? 1.f : th.om);
    const float2 om1 = make_float2(bnd0 ? 0.f : th.om1, bnd1 ? 0.f : th.om1);
    const float2 usq = mul2(f2(1.5f), fma2(ux, ux, fma2(uy, uy, mul2(uz, uz))));
    const float2 nusq = mul2(f2(-1.f), usq);
    // om w rho and om w drho for the two weight classes of the moving
    // populations and the rest population; om 3 w rho for the odd part
    const float2 omrho = mul2(om, rho), omdrho = mul2(om, drho);
    const float2 r18 = mul2(f2(1.f / 18.f), omrho), d18 = mul2(f2(1.f / 18.f), omdrho);
    const float2 r36 = mul2(f2(1.f / 36.f), omrho), d36 = mul2(f2(1.f / 36.f), omdrho);
    const float2 t18 = mul2(f2(3.f / 18.f), omrho), t36 = mul2(f2(3.f / 36.f), omrho);
    float2 sfr, srcw[2], ua;
    if (ACCEL) {  // Guo source: (1 - om/2) w rho (3 (c.a - u.a) + 9 (c.u)(c.a)), zero on boundary lanes
        const float2 sf = make_float2(bnd0 ? 0.f : th.srcfac, bnd1 ? 0.f : th.srcfac);
        sfr = mul2(sf, rho);
        srcw[0] = mul2(sfr, f2(1.f / 18.f));
        srcw[1] = mul2(sfr, f2(1.f / 36.f));
        ua = fma2(ux, ac[0], fma2(uy, ac[1], mul2(uz, ac[2])));
    }
    E* out = Bb + s;
    // population 0: om w0 (drho - rho usq)
    {
        const float2 odeq = mul2(f2(1.f / 3.f), fma2(omrho, nusq, omdrho));
        float2 val = fma2(om1, f[0], odeq);
        if (ACCEL) val = fma2(sfr, make_float2(-ua.x, -ua.y), val);  // (1 - om/2) w0 rho 3 (-u.a), 3 w0 = 1
        if (act) IO::store(out, val);
    }
#pragma unroll
    for (int i = 1; i < kQ; i += 2) {
        out += i == 1 ? n3 : 2 * n3;  // row of population i; population i + 1 is one row further
        const int cx = cvec(i, 0), cy = cvec(i, 1), cz = cvec(i, 2);
        const bool w18 = i < 7;
        float2 cu;
        if (cx && cy) cu = cy > 0 ? (cx > 0 ? add2(ux, uy) : make_float2(-(ux.x + uy.x), -(ux.y + uy.y))) : (cx > 0 ? sub2(ux, uy) : sub2(uy, ux));
        else if (cx && cz) cu = cz > 0 ? (cx > 0 ? add2(ux, uz) : make_float2(-(ux.x + uz.x), -(ux.y + uz.y))) : (cx > 0 ? sub2(ux, uz) : sub2(uz, ux));
        else if (cy && cz) cu = cz > 0 ? (cy > 0 ? add2(uy, uz) : make_float2(-(uy.x + uz.x), -(uy.y + uz.y))) : (cy > 0 ? sub2(uy, uz) : sub2(uz, uy));
        else cu = cx ? ux : (cy ? uy : uz);  // axis pairs: c_i = +x, +y or +z for odd i
        // om (w (drho + rho (4.5 cu^2 - usq))) and om (3 w rho cu)
        const float2 t = fma2(mul2(f2(4.5f), cu), cu, nusq);
        const float2 oeven = fma2(w18 ? r18 : r36, t, w18 ? d18 : d36);
        const float2 oodd = mul2(w18 ? t18 : t36, cu);
        float2 vp = fma2(om1, f[i], add2(oeven, oodd));
        float2 vm = fma2(om1, f[i + 1], sub2(oeven, oodd));
        if (ACCEL) {
            float ca = 0.f;  // c_i . a (uniform per box)
            if (cx) ca += cx * (float)bd.accel[0];
            if (cy) ca += cy * (float)bd.accel[1];
            if (cz) ca += cz * (float)bd.accel[2];
            const float2 sw = w18 ? srcw[0] : srcw[1];
            // + : 3 (ca - ua) + 9 cu ca ;  - : 3 (-ca - ua) + 9 cu ca  (c -> -c flips ca and cu)
            const float2 nine_cu_ca = mul2(f2(9.f * ca), cu);
            const float2 sp = fma2(f2(3.f), sub2(f2(ca), ua), nine_cu_ca);
            const float2 sm = fma2(f2(3.f), sub2(f2(-ca), ua), nine_cu_ca);
            vp = fma2(sw, sp, vp);
            vm = fma2(sw, sm, vm);
        }
        if (act) {
            IO::store(out, vp);
            IO::store(out + n3, vm);
        }
    }
}

// Consumer body of a box with the fluctuating collision (lbt_fluct.cuh): the
// thread's sites (the adjacent pair s0 + 2c, s0 + 2c + 1 when SPT = 2, site
// s0 + c when SPT = 1) pulled into registers, the stage released, then site by
// site the moments and either the boundary equilibrium or the fluctuating
// collision with the site's Philox noise of step n.  Boxes with a body force
// or a chain do not take this path.
template <int ST, int SPT, bool PER>
__device__ __forceinline__ void staged_tile_fluct(const SCParams& p, const StagedTile<ST>& th,
                                                  const unsigned char* stage, uint64_t* empty, int64_t n)
{
    using S = Stor<ST>;
    using E = typename S::E;
    using A = typename S::A;
    using R = typename S::R;
    constexpr int H = Staged<ST, SPT>::kHalo;
    const int tid = threadIdx.x;
    const int s0 = (int)th.s0;
    const BoxDev& bd = th.bd;
    const int Ei = bd.E;
    const int n3 = (int)bd.n3;
    const int per = bd.per_mask;
    const bool px = per & 1, py = per & 2, pz = per & 4;
    const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
    E* Bb = reinterpret_cast<E*>(p.B) + bd.f_off;
    auto local = [&](int k) { return SPT == 2 ? 2 * tid + k : tid; };

    int xs_[SPT], ys_[SPT], zs_[SPT];
    bool act[SPT], bnd[SPT];
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        const int s = s0 + local(k);
        act[k] = s < n3;
        const int sc = act[k] ? s : 0;
        const int row = div_e(sc, bd.div_magic);
        xs_[k] = sc - row * Ei;
        zs_[k] = div_e(row, bd.div_magic);
        ys_[k] = row - zs_[k] * Ei;
        bnd[k] = act[k] && ((!px && (xs_[k] == 0 || xs_[k] == Ei - 1)) || (!py && (ys_[k] == 0 || ys_[k] == Ei - 1)) ||
                            (!pz && (zs_[k] == 0 || zs_[k] == Ei - 1)));
    }
    A f[kQ][SPT];
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        const int cx = cvec(i, 0), cy = cvec(i, 1), cz = cvec(i, 2);
        const E* row = reinterpret_cast<const E*>(stage + i * Staged<ST, SPT>::kRowStride);
#pragma unroll
        for (int k = 0; k < SPT; k++) {
            A v = S::in(row[H + local(k) - cx]);
            if (PER) {
                const int xs = xs_[k] - cx, ys = ys_[k] - cy, zs = zs_[k] - cz;
                const bool wrap = (px && (xs < 0 || xs >= Ei)) || (py && (ys < 0 || ys >= Ei)) ||
                                  (pz && (zs < 0 || zs >= Ei));
                if (wrap && act[k])
                    v = S::in(Ab[(int64_t)i * n3 + ((int64_t)wrapi(zs, Ei) * Ei + wrapi(ys, Ei)) * Ei + wrapi(xs, Ei)]);
            }
            f[i][k] = (act[k] && !bnd[k]) ? v : A(0);
        }
    }
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(empty);  // this warp is done with the stage

    const FluctDev& fd = p.fluct[th.box];
    bool nonfinite = false;
#pragma unroll
    for (int k = 0; k < SPT; k++) {
        A d[kQ], r = A(0), jx = A(0), jy = A(0), jz = A(0);
#pragma unroll
        for (int i = 0; i < kQ; i++) {
            d[i] = f[i][k];
            r += d[i];
            if (cvec(i, 0)) jx += cvec(i, 0) * d[i];
            if (cvec(i, 1)) jy += cvec(i, 1) * d[i];
            if (cvec(i, 2)) jz += cvec(i, 2) * d[i];
        }
        const A rho = A(1) + r;
        nonfinite |= !(rho > A(0) && rho < A(1e30));
        A out[kQ];
        if (bnd[k]) {  // boundary equilibrium of the boundary velocity, as in the BGK bodies
            TimeWeights<R> tw;
#pragma unroll
            for (int a = 0; a < 4; a++) {
                tw.slot[a] = th.slot[a];
                tw.c[a] = th.c[a];
            }
            int pp, qq;
            const int fc = owning_face(xs_[k], ys_[k], zs_[k], Ei, per, pp, qq);
            R ub[3];
            boundary_velocity<R>(reinterpret_cast<const R*>(p.ring), p.ring_slot_elems, bd, fc, pp, qq, tw, ub);
            const A dr = th.drho_b, rb = A(1) + dr;
            const A u0 = (A)ub[0], u1 = (A)ub[1], u2 = (A)ub[2];
            const A usq = A(1.5) * (u0 * u0 + u1 * u1 + u2 * u2);
#pragma unroll
            for (int i = 0; i < kQ; i++) {
                A cu = A(0);
                if (cvec(i, 0)) cu += cvec(i, 0) * u0;
                if (cvec(i, 1)) cu += cvec(i, 1) * u1;
                if (cvec(i, 2)) cu += cvec(i, 2) * u2;
                out[i] = wgt<A>(i) * (dr + rb * (A(3) * cu + A(4.5) * cu * cu - usq));
            }
        } else {
            const A inv = A(1) / rho;
            fluct_collide<A>(d, r, jx * inv, jy * inv, jz * inv, fd, n, s0 + local(k), out);
        }
        if (act[k]) {
            E* o = Bb + s0 + local(k);
#pragma unroll
            for (int i = 0; i < kQ; i++) o[(int64_t)i * n3] = S::out(out[i]);
        }
    }
    if (__any_sync(0xffffffffu, nonfinite) && (tid & 31) == 0) atomicCAS(&p.status[th.box], 0, LB_ERR_NONFINITE);
}

// Consumer warps: take the stages in order until the producer posts the end.
// KIND 0: every box of the launch is non-periodic and force-free, so only
// that tile body is compiled in (fewer registers than the kernel that carries
// all bodies).
template <int ST, int SPT, int KIND>
__device__ __forceinline__ void staged_consume(const SCParams& p, unsigned char* smem, StagedHeader<ST>* hd,
                                               int64_t n)
{
    constexpr bool GENERAL = KIND > 0;
    using G = Staged<ST, SPT>;
    using E = typename Stor<ST>::E;
    for (int k = 0;; k++) {
        const int st = k % G::kStages;
        const uint32_t phase = (uint32_t)((k / G::kStages) & 1);
        const bool arrived = mbar_wait_bounded(&hd->full[st], phase, p.wait_ns);
        if (!__all_sync(0xffffffffu, arrived)) {
            // nothing arrived within the limit: flag the box, let copies still
            // in flight land (one more bounded wait) and leave
            if ((threadIdx.x & 31) == 0) {
                const int b = *reinterpret_cast<volatile const int32_t*>(&hd->t[k % (2 * G::kStages)].box);
                atomicCAS(&p.status[b >= 0 && b < p.nboxes ? b : 0], 0, LB_ERR_TIMEOUT);
            }
            mbar_wait_bounded(&hd->full[st], phase, p.wait_ns);
            return;
        }
        const StagedTile<ST>& th = hd->t[k % (2 * G::kStages)];
        const int b = th.box;
        if (b < 0) return;  // end of work
        const int64_t s0 = th.s0;
        const BoxDev& bd = th.bd;
        const unsigned char* stage = smem + kStagedHeaderBytes + st * G::kStageBytes;
        if (th.frozen) {
            // frozen box: release the stage, the state does not change
            __syncwarp();
            if ((threadIdx.x & 31) == 0) mbar_arrive(&hd->empty[st]);
            const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
            E* Bb = reinterpret_cast<E*>(p.B) + bd.f_off;
            for (int t = threadIdx.x; t < G::kSites; t += kStagedConsumers)
                if (s0 + t < bd.n3)
                    for (int i = 0; i < kQ; i++) Bb[(int64_t)i * bd.n3 + s0 + t] = Ab[(int64_t)i * bd.n3 + s0 + t];
        } else if (KIND == 2 && bd.fluct) {
            if constexpr (KIND == 2) {
                if (bd.per_mask) staged_tile_fluct<ST, SPT, true>(p, th, stage, &hd->empty[st], n);
                else staged_tile_fluct<ST, SPT, false>(p, th, stage, &hd->empty[st], n);
            }
        } else if constexpr (SPT == 2 && ST != kF64) {  // adjacent site pairs, packed FP32
            if (!GENERAL) {
                staged_tile_pair<ST, false, false>(p, th, stage, &hd->empty[st]);
            } else if (bd.per_mask == 0) {
                if (bd.has_accel) staged_tile_pair<ST, false, true>(p, th, stage, &hd->empty[st]);
                else staged_tile_pair<ST, false, false>(p, th, stage, &hd->empty[st]);
            } else {
                if (bd.has_accel) staged_tile_pair<ST, true, true>(p, th, stage, &hd->empty[st]);
                else staged_tile_pair<ST, true, false>(p, th, stage, &hd->empty[st]);
            }
        } else if (!GENERAL) {
            staged_tile<ST, SPT, false, false>(p, th, stage, &hd->empty[st]);
        } else if (bd.per_mask == 0) {
            if (bd.has_accel) staged_tile<ST, SPT, false, true>(p, th, stage, &hd->empty[st]);
            else staged_tile<ST, SPT, false, false>(p, th, stage, &hd->empty[st]);
        } else {
            if (bd.has_accel) staged_tile<ST, SPT, true, true>(p, th, stage, &hd->empty[st]);
            else staged_tile<ST, SPT, true, false>(p, th, stage, &hd->empty[st]);
        }
    }
}

// Prefetch into L2 (evict-last) of the upsampler residuals of substep ms for
// the boundary sites of the box rows that tile [s0, s0 + T) covers: the
// x-face sites at both ends of every row (faces 0 and 1, in-face (y, z)) and
// whole rows on a y or z face, three components each.  One row per lane;
// every address lies inside the box's residual columns.
__device__ __forceinline__ void prefetch_l2(const float* a)
{
    asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(a));
}
__device__ __forceinline__ void prefetch_mlp_residuals(const SCParams& p, const BoxDev& bd, int ms, int64_t s0, int T,
                                                       int lane)
{
    const int Eb = bd.E;
    const int64_t fe = (int64_t)Eb * Eb, str = p.mlp_ystride;
    const float* y0 = p.mlp_y + (int64_t)(3 * (ms - 1)) * str + bd.mlp_row;
    const int64_t r_first = s0 / Eb, r_end = (s0 + T - 1) / Eb + 1;
    for (int64_t r = r_first + lane; r < r_end && r < fe; r += 32) {
        const int yy = (int)(r % Eb), zz = (int)(r / Eb);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            prefetch_l2(y0 + c * str + (int64_t)zz * Eb + yy);       // x- face
            prefetch_l2(y0 + c * str + fe + (int64_t)zz * Eb + yy);  // x+ face
        }
        const int fo = yy == 0 ? 2 : (yy == Eb - 1 ? 3 : (zz == 0 ? 4 : (zz == Eb - 1 ? 5 : -1)));
        if (fo >= 0) {
            const int q = fo < 4 ? zz : yy;  // in-face (x, z) on a y face, (x, y) on a z face
            const float* row = y0 + fo * fe + (int64_t)q * Eb;
            for (int x0 = 0; x0 < Eb; x0 += 32)
#pragma unroll
                for (int c = 0; c < 3; c++) prefetch_l2(row + c * str + x0);
        }
    }
}

// Producer warp (the last warp): claims tiles from the global counter (reset
// to zero by the forced re-collision at the end of every step, so a block that
// starts late -- its SM still busy with the bead kernel -- simply takes fewer
// tiles) and fills the stages as the consumers free them.  Lane 0 claims,
// waits for the stage and writes the tile header; lane i < 19 handles
// population row i: its source range, the zeroing of the part of the row that
// lies outside the box's arrays (those sites are boundary sites: their pulled
// values are multiplied by zero and must be finite, so no consumer may read
// what a previous tile left there), and its bulk copy.
template <int ST, int SPT, int KIND>
__device__ __forceinline__ void staged_produce(const SCParams& p, unsigned char* smem, StagedHeader<ST>* hd, int64_t n)
{
    using G = Staged<ST, SPT>;
    using E = typename Stor<ST>::E;
    using R = typename Stor<ST>::R;
    using A = typename Stor<ST>::A;
    constexpr int T = G::kSites, H = G::kHalo, W = T + 2 * H;
    const int lane = threadIdx.x & 31;
    int cy = 0, cz = 0;  // y and z components of this lane's population
#pragma unroll
    for (int i = 0; i < kQ; i++)
        if (lane == i) {
            cy = cvec(i, 1);
            cz = cvec(i, 2);
        }
    const uint64_t pol = p.hint_loads ? l2_evict_first_policy() : 0;
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(p.tile_counter);
    long long next = lane == 0 ? (long long)atomicAdd(ctr, 1ull) : 0;
    next = __shfl_sync(0xffffffffu, next, 0);
    int last_b = -1;
    TimeWeights<R> tw{};
    int mlp_s = 0;
    for (int k = 0;; k++) {
        const int st = k % G::kStages;
        // the stage's previous tile must be released by all consumer warps; if
        // that does not happen within the limit the consumers have left
        if (k >= G::kStages) {
            bool ok = true;
            if (lane == 0) ok = mbar_wait_bounded(&hd->empty[st], (uint32_t)(((k / G::kStages) - 1) & 1), p.wait_ns);
            if (!__shfl_sync(0xffffffffu, ok, 0)) return;
        }
        const int64_t t = next;
        StagedTile<ST>& th = hd->t[k % (2 * G::kStages)];
        if (t >= p.total_tiles) {
            if (lane == 0) {
                th.box = -1;
                mbar_arrive(&hd->full[st]);  // completes the phase with no bytes: end of work
            }
            // no tile left for this block: the kernel after this one (the
            // forced re-collision, a programmatic dependent) may be scheduled
            // once every block has got here; it waits on the device for this
            // grid to complete
            asm volatile("griddepcontrol.launch_dependents;");
            return;
        }
        if (lane == 0) next = (long long)atomicAdd(ctr, 1ull);  // the next claim overlaps this tile's copies
        const int b = locate_box_warp(p, t, lane);
        const BoxDev& bd = p.boxes[b];
        const int64_t s0 = (t - p.tile_prefix[b]) * T;
        // header: the box record word by word across the lanes, the rest by lane 0
        static_assert(sizeof(BoxDev) % 8 == 0 && sizeof(BoxDev) / 8 <= 32, "box record copied by one warp");
        if (lane < (int)(sizeof(BoxDev) / 8))
            reinterpret_cast<uint64_t*>(&th.bd)[lane] = reinterpret_cast<const uint64_t*>(&bd)[lane];
        __syncwarp();
        if (lane == 0) {
            if (b != last_b) {  // boundary-layer constants of this box at step n
                tw = time_weights<R>(n, bd.K, bd.time_interp, p.ring_slots);
                mlp_s = bd.mlp_row >= 0 ? mlp_substep(n, bd.K) : 0;
                last_b = b;
            }
            if (KIND > 0 && bd.frame) {  // the header carries the body acceleration of step n (frame
                                         // boxes carry a body force, so they run a general kernel)
                double a[3];
                frame_accel_at(bd, p.faccel, p.ring_slots, n, a);
                for (int c = 0; c < 3; c++) th.bd.accel[c] = a[c];
            }
            th.box = b;
            th.s0 = s0;
            th.mlp_s = mlp_s;
            th.frozen = p.status[b] != 0;
            for (int a = 0; a < 4; a++) {
                th.slot[a] = tw.slot[a];
                th.c[a] = tw.c[a];
            }
            th.om = A(1) / (A)bd.tau;
            th.om1 = A(1) - th.om;
            th.srcfac = A(1) - A(0.5) * th.om;
            th.drho_b = (A)bd.rho_b - A(1);
        }
        // row `lane`: source range clamped to the box's arrays
        unsigned char* stage = smem + kStagedHeaderBytes + st * G::kStageBytes;
        const int64_t Ei = bd.E, n3 = bd.n3;
        const int64_t start = s0 - (cy * Ei + cz * Ei * Ei) - H;
        const int64_t lo = start > 0 ? start : 0;
        const int64_t hi = start + W < n3 ? start + W : n3;
        const bool mine = lane < kQ && hi > lo;
        uint32_t bytes = mine ? (uint32_t)((hi - lo) * sizeof(E)) : 0u;
        if (lane < kQ) {
            const int a = mine ? (int)(lo - start) : W;  // first copied element
            const int e = mine ? (int)(hi - start) : W;  // end of the copied elements
            if (a > 0 || e < W) {
                uint4* row = reinterpret_cast<uint4*>(stage + lane * G::kRowStride);
                constexpr int per16 = 16 / (int)sizeof(E);
                for (int x = 0; x < a; x += per16) row[x / per16] = make_uint4(0, 0, 0, 0);
                for (int x = e; x < W; x += per16) row[x / per16] = make_uint4(0, 0, 0, 0);
            }
        }
        uint32_t total = bytes;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
        next = __shfl_sync(0xffffffffu, next, 0);
        __syncwarp();  // header and zeroed parts written before the stage is armed
        if (t == p.withhold_tile) {
            // test only: this stage is never armed and no copy is issued, so
            // its full barrier never completes and the consumers' bounded wait
            // runs out (the header above is in place for them to name the box)
            __threadfence_block();
            continue;
        }
        if (lane == 0) mbar_arrive_expect_tx(&hd->full[st], total);
        __syncwarp();
        if (mine) {
            fence_proxy_async_smem();
            const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
            if (p.hint_loads)
                bulk_load_hint(stage + lane * G::kRowStride + (lo - start) * sizeof(E), Ab + (int64_t)lane * n3 + lo,
                               bytes, &hd->full[st], pol);
            else
                bulk_load(stage + lane * G::kRowStride + (lo - start) * sizeof(E), Ab + (int64_t)lane * n3 + lo, bytes,
                          &hd->full[st]);
        }
        // upsampler boxes: the residuals the tile's boundary sites will add
        // come from an output far larger than L2; prefetch them into L2 while
        // the copies are in flight, so that the consumers' loads hit there
        const int ms = __shfl_sync(0xffffffffu, mlp_s, 0);
        if (bd.mlp_row >= 0 && ms > 0) prefetch_mlp_residuals(p, bd, ms, s0, T, lane);
    }
}

// KIND 0: every box of the launch is plain (velocity faces, no body force);
// 1: some box is periodic or carries a body force; 2: some box also takes the
// fluctuating collision.  Each kind compiles only the tile bodies it can meet.
template <int ST, int SPT, int KIND>
__global__ void __launch_bounds__(kStagedThreads, 1) k_stream_collide_staged(SCParams p)
{
    using G = Staged<ST, SPT>;
    extern __shared__ __align__(128) unsigned char smem[];
    StagedHeader<ST>* hd = reinterpret_cast<StagedHeader<ST>*>(smem);
    if (threadIdx.x == 0) {
        for (int st = 0; st < G::kStages; st++) {
            mbar_init(&hd->full[st], 1);
            mbar_init(&hd->empty[st], kStagedConsumerWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();
    // Launched as a programmatic dependent of the kernel before it on the
    // stream (the previous step's forced re-collision): the block may start
    // while that kernel runs, and everything above touched only shared
    // memory.  Wait here for it to complete and its writes to be visible.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t n = *p.step;
    if (threadIdx.x >= kStagedConsumers) {
        staged_produce<ST, SPT, KIND>(p, smem, hd, n);  // the whole last warp
        return;
    }
    staged_consume<ST, SPT, KIND>(p, smem, hd, n);
}

}  // namespace lbt
