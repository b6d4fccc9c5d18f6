// Kernel templates of the tracer-box lattice Boltzmann step.  Included once
// per storage format by lbt_inst_*.cu.
//
// One step n -> n+1 (state A = post-collision populations of step n, with the
// boundary layer at the equilibrium of t = n):
//   k_bead_couple     (side stream)  chain MD over the step, force list
//   k_stream_collide                  every site of every box: pull, BGK
//                                     collide (interior) or boundary
//                                     equilibrium at t = n+1, write B
//   k_forced                          re-collide the forced sites with the
//                                     bead force, advance the step counter
#pragma once
#include <type_traits>

#include "lbt_device.cuh"
#include "lbt_sc_staged.cuh"

namespace lbt {

// ---------------------------------------------------------------------------
// Fused stream-collide + boundary layer.
//
// Work unit: a group of VW consecutive x-sites, moved with one vector load per
// population.  Groups of a box are numbered linearly in memory order, a tile
// is blockDim.x consecutive groups of one box, and blocks walk the global tile
// list (all boxes) with a stride of gridDim.x (persistent when the grid is
// smaller than the tile count).
//
// Pull scheme: population i of site x comes from x - c_i.  The y/z shift moves
// whole rows, so the load stays aligned; the x shift (c_ix = +-1) needs one
// element of the neighbouring group, taken from the neighbouring lane by a
// warp shuffle, or loaded directly at a warp edge and at a periodic x wrap.
// ---------------------------------------------------------------------------
template <int ST, int VW, bool ACCEL>
__device__ __forceinline__ void sc_tile(const SCParams& p, const BoxDev& bd, const double acc[3], int64_t G, int64_t n,
                                        int lane)
{
    using S = Stor<ST>;
    using E = typename S::E;
    using A = typename S::A;
    using R = typename S::R;
    using P = Pack<E, VW>;
    using Raw = typename P::Raw;

    const int Ei = bd.E;
    const int64_t n3 = bd.n3;
    const int gpr = Ei / VW;
    // body acceleration of the step in the arithmetic type, converted once
    const A acA[3] = {(A)acc[0], (A)acc[1], (A)acc[2]};
    const int64_t groups = n3 / VW;
    const bool active = G < groups;
    const int64_t Gc = active ? G : 0;
    const int xg = (int)(Gc % gpr);
    const int64_t row = Gc / gpr;
    const int y = (int)(row % Ei);
    const int z = (int)(row / Ei);
    const int per = bd.per_mask;
    const bool px = per & 1, py = per & 2, pz = per & 4;
    const bool row_bnd = (!py && (y == 0 || y == Ei - 1)) || (!pz && (z == 0 || z == Ei - 1));
    const bool interior = active && !row_bnd;

    const E* Ab = reinterpret_cast<const E*>(p.A) + bd.f_off;
    E* Bb = reinterpret_cast<E*>(p.B) + bd.f_off;

    // ---- loads ----
    P v[kQ];
    A nb[kQ];
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        int ys = y - cvec(i, 1), zs = z - cvec(i, 2);
        if (py) ys = wrapi(ys, Ei);
        if (pz) zs = wrapi(zs, Ei);
        const int64_t src = ((int64_t)zs * Ei + ys) * gpr + xg;
        v[i].raw = interior ? ld_nc(reinterpret_cast<const Raw*>(Ab + (int64_t)i * n3) + src) : zero_raw<Raw>();
    }
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        const int cx = cvec(i, 0);
        if (cx == 0) continue;
        int ys = y - cvec(i, 1), zs = z - cvec(i, 2);
        if (py) ys = wrapi(ys, Ei);
        if (pz) zs = wrapi(zs, Ei);
        const E* rowp = Ab + (int64_t)i * n3 + ((int64_t)zs * Ei + ys) * Ei;
        if (cx == 1) {
            // site x0 needs element x0 - 1: last element of the previous group
            A t = __shfl_up_sync(0xffffffffu, S::in(v[i].e[VW - 1]), 1);
            const bool need = interior && (xg == 0 ? px : lane == 0);
            if (need) t = S::in(rowp[xg == 0 ? Ei - 1 : xg * VW - 1]);
            nb[i] = t;
        } else {
            // site x0 + VW - 1 needs element x0 + VW: first element of the next group
            A t = __shfl_down_sync(0xffffffffu, S::in(v[i].e[0]), 1);
            const bool need = interior && (xg == gpr - 1 ? px : lane == 31);
            if (need) t = S::in(rowp[xg == gpr - 1 ? 0 : (xg + 1) * VW]);
            nb[i] = t;
        }
    }

    // ---- moments of the pulled populations ----
    auto fval = [&](int i, int k) -> A {
        const int cx = cvec(i, 0);
        if (cx == 0) return S::in(v[i].e[k]);
        if (cx == 1) return k == 0 ? nb[i] : S::in(v[i].e[k - 1]);
        return k == VW - 1 ? nb[i] : S::in(v[i].e[k + 1]);
    };

    A drho[VW], ux[VW], uy[VW], uz[VW];
    bool nonfinite = false;  // a density that is not finite or not positive
#pragma unroll
    for (int k = 0; k < VW; k++) {
        A r = A(0), jx = A(0), jy = A(0), jz = A(0);
#pragma unroll
        for (int i = 0; i < kQ; i++) {
            const A f = fval(i, k);
            r += f;
            if (cvec(i, 0)) jx += cvec(i, 0) * f;
            if (cvec(i, 1)) jy += cvec(i, 1) * f;
            if (cvec(i, 2)) jz += cvec(i, 2) * f;
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
    // flag the box (it freezes from the next step on); sites that pulled no
    // populations (boundary rows, inactive groups) hold zeros and never raise it
    if (__any_sync(0xffffffffu, nonfinite) && lane == 0) atomicCAS(&p.status[bd.box], 0, LB_ERR_NONFINITE);

    // ---- boundary sites: equilibrium of the interpolated boundary velocity ----
    unsigned bmask = 0;
    if (active) {
        if (row_bnd) bmask = (1u << VW) - 1u;
        else if (!px) bmask = (xg == 0 ? 1u : 0u) | (xg == gpr - 1 ? (1u << (VW - 1)) : 0u);
    }
    if (bmask) {
        const TimeWeights<R> tw = time_weights<R>(n, bd.K, bd.time_interp, p.ring_slots);
        const int s_mlp = bd.mlp_row >= 0 ? mlp_substep(n, bd.K) : 0;
        const R* ring = reinterpret_cast<const R*>(p.ring);
#pragma unroll
        for (int k = 0; k < VW; k++) {
            if (bmask & (1u << k)) {
                int pp, qq;
                const int x = xg * VW + k;
                const int f = owning_face(x, y, z, Ei, per, pp, qq);
                float res[3];
                load_mlp_residual(p, bd, s_mlp, f, pp, qq, res);
                R ub[3];
                boundary_velocity<R>(ring, p.ring_slot_elems, bd, f, pp, qq, tw, ub);
                add_mlp_residual<R>(p, bd, res, ub);
                drho[k] = (A)bd.rho_b - A(1);
                ux[k] = (A)ub[0];
                uy[k] = (A)ub[1];
                uz[k] = (A)ub[2];
            }
        }
    }

    // ---- collide and store, one population at a time ----
    const A om = A(1) / (A)bd.tau;
    const A srcfac = A(1) - A(0.5) * om;
    A usq[VW], ua[VW];
#pragma unroll
    for (int k = 0; k < VW; k++) {
        usq[k] = A(1.5) * (ux[k] * ux[k] + uy[k] * uy[k] + uz[k] * uz[k]);
        if (ACCEL) ua[k] = ux[k] * acA[0] + uy[k] * acA[1] + uz[k] * acA[2];
    }
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        const A w = wgt<A>(i);
        const int cx = cvec(i, 0), cy = cvec(i, 1), cz = cvec(i, 2);
        P o;
#pragma unroll
        for (int k = 0; k < VW; k++) {
            const A rho = A(1) + drho[k];
            A cu = A(0);
            if (cx) cu += cx * ux[k];
            if (cy) cu += cy * uy[k];
            if (cz) cu += cz * uz[k];
            const A deq = w * (drho[k] + rho * (A(3) * cu + A(4.5) * cu * cu - usq[k]));
            const A f = fval(i, k);
            A val = f + om * (deq - f);
            if (ACCEL) {
                A ca = A(0);  // c_i . a in the arithmetic type (FP64 is slow on this part)
                if (cx) ca += cx * acA[0];
                if (cy) ca += cy * acA[1];
                if (cz) ca += cz * acA[2];
                val += srcfac * w * rho * (A(3) * (ca - ua[k]) + A(9) * cu * ca);
            }
            if (bmask & (1u << k)) val = deq;
            o.e[k] = S::out(val);
        }
        if (active) reinterpret_cast<Raw*>(Bb + (int64_t)i * n3)[G] = o.raw;
    }
}

template <int ST, int VW>
__device__ __forceinline__ void copy_tile(const SCParams& p, const BoxDev& bd, int64_t G)
{
    using E = typename Stor<ST>::E;
    using Raw = typename Pack<E, VW>::Raw;
    if (G >= bd.n3 / VW) return;
    const Raw* a = reinterpret_cast<const Raw*>(reinterpret_cast<const E*>(p.A) + bd.f_off);
    Raw* b = reinterpret_cast<Raw*>(reinterpret_cast<E*>(p.B) + bd.f_off);
    const int64_t gq = bd.n3 / VW;
    for (int i = 0; i < kQ; i++) b[i * gq + G] = a[i * gq + G];
}

template <int ST, int VW>
__global__ void __launch_bounds__(256) k_stream_collide(SCParams p)
{
    const int lane = threadIdx.x & 31;
    const int64_t n = *p.step;
    for (int64_t tile = blockIdx.x; tile < p.total_tiles; tile += gridDim.x) {
        int lo = 0, hi = p.nboxes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.tile_prefix[mid] <= tile) lo = mid;
            else hi = mid - 1;
        }
        const BoxDev& bd = p.boxes[lo];
        const int64_t G = (tile - p.tile_prefix[lo]) * blockDim.x + threadIdx.x;
        if (p.status[lo] != 0) {
            copy_tile<ST, VW>(p, bd, G);  // frozen box: state does not change
            continue;
        }
        double acc[3];
        frame_accel_at(bd, p.faccel, p.ring_slots, n, acc);  // body acceleration of step n
        if (bd.has_accel) sc_tile<ST, VW, true>(p, bd, acc, G, n, lane);
        else sc_tile<ST, VW, false>(p, bd, acc, G, n, lane);
    }
}

// ---------------------------------------------------------------------------
// Per-site helpers for the scalar kernels (bead gather, forced re-collision,
// fields).
// ---------------------------------------------------------------------------
template <int ST>
__device__ __forceinline__ void pull_site(const typename Stor<ST>::E* Ab, int64_t n3, int E, int per, int x, int y,
                                          int z, typename Stor<ST>::A f[kQ])
{
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        int xs = x - cvec(i, 0), ys = y - cvec(i, 1), zs = z - cvec(i, 2);
        if (per & 1) xs = wrapi(xs, E);
        if (per & 2) ys = wrapi(ys, E);
        if (per & 4) zs = wrapi(zs, E);
        f[i] = Stor<ST>::in(Ab[(int64_t)i * n3 + ((int64_t)zs * E + ys) * E + xs]);
    }
}

template <class A>
__device__ __forceinline__ void moments(const A f[kQ], A& drho, A j[3])
{
    drho = A(0);
    j[0] = j[1] = j[2] = A(0);
#pragma unroll
    for (int i = 0; i < kQ; i++) {
        drho += f[i];
        if (cvec(i, 0)) j[0] += cvec(i, 0) * f[i];
        if (cvec(i, 1)) j[1] += cvec(i, 1) * f[i];
        if (cvec(i, 2)) j[2] += cvec(i, 2) * f[i];
    }
}

// ---------------------------------------------------------------------------
// Bead coupling: one block per chain, one thread per bead in the MD phase.
//
// Chain model: Kremer-Grest bead-spring chain (FENE bonds plus WCA repulsion
// between all pairs), coupled to the fluid by Stokes friction.  Positions are
// FP64; forces, velocities and the momentum handed to the fluid use MT
// (double for FP64 storage, float otherwise), with pair geometry taken from
// positions relative to bead 0's start-of-step position.  WCA pairs come from
// a Verlet list in shared memory, rebuilt whenever a bead has moved more than
// half the skin since the last build, so no pair within the cut-off is missed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int32_t* st, int code) { atomicCAS(st, 0, code); }

constexpr int kMaxTasks = 48;           // pair tasks (bonds + Verlet neighbours) per bead
constexpr int kMaxStencilNb = 24;       // listed beads with a nearby stencil (more: scan all)
constexpr int kNoiseChunk = 64;         // substeps whose noise is drawn at once (at most)
constexpr int kBeadThreadsMax = 2 * kMaxBeads;  // 512: two MD lanes per bead at the largest chain
constexpr size_t kBeadDynMax = 160 * 1024;      // dynamic shared memory budget of the bead kernel

template <class MT>
struct Vec4;
template <>
struct Vec4<float> {
    using T = float4;
};
template <>
struct Vec4<double> {
    struct __align__(32) T {
        double x, y, z, w;
    };
};

// Noise chunk of the bead kernel for chains of at most maxb beads: as many
// substeps (at most kNoiseChunk) as fit the dynamic shared-memory budget next
// to the two position buffers, all 4-vectors.
template <class MT>
inline int bead_noise_chunk(int maxb)
{
    const size_t per = 4 * sizeof(MT) * (size_t)(maxb > 0 ? maxb : 1);
    const int c = (int)(kBeadDynMax / per) - 2;
    return c < kNoiseChunk ? (c < 1 ? 1 : c) : kNoiseChunk;
}

// Dynamic shared memory: positions relative to bead 0's start-of-step
// position, double-buffered over substeps, and the noise of one chunk.
template <class MT>
inline size_t bead_dyn_bytes(int maxb)
{
    return 4 * sizeof(MT) * (size_t)maxb * (2 + bead_noise_chunk<MT>(maxb));
}

// Pair-force constants of a chain in the MD precision.
template <class MT>
struct PairConsts {
    MT R02, inv_R02, kf, sig2, rc2, e24;
};

// Pair force on a bead at X from the partner at q, added to F, in one code
// path for both laws (force = fac (X - q)):
//   FENE: fac = -k / (1 - r^2/R0^2)
//   WCA:  fac = 24 eps (2 (s/r)^12 - (s/r)^6) / r^2, r < 2^(1/6) s
// Both beads of a pair evaluate the same r^2 from exactly negated
// differences, so the two forces cancel exactly.  Returns true for a bond
// stretched to R0 or beyond.
template <class MT>
__device__ __forceinline__ bool pair_force(const MT X[3], const typename Vec4<MT>::T& q, bool fene,
                                           const PairConsts<MT>& c, MT F[3])
{
    const MT rx = X[0] - q.x, ry = X[1] - q.y, rz = X[2] - q.z;
    const MT r2 = rx * rx + ry * ry + rz * rz;
    const MT inv = recip(fene ? MT(1) - r2 * c.inv_R02 : r2);
    const MT s2 = c.sig2 * inv, s6 = s2 * s2 * s2;
    const MT fac = fene ? -c.kf * inv : (r2 < c.rc2 ? c.e24 * (MT(2) * s6 * s6 - s6) * inv : MT(0));
    F[0] += fac * rx;
    F[1] += fac * ry;
    F[2] += fac * rz;
    return fene && r2 >= c.R02;
}

// Noise of substeps c0 .. c0 + nc - 1 for all N beads (three unit-variance
// uniforms per bead and substep, Philox4x32-10 with counter (step, substep,
// bead, box) and the chain seed as key), spread over the block's threads.
template <class MT>
__device__ __forceinline__ void md_noise(typename Vec4<MT>::T* sXi, int64_t n, int c0, int nc, int N, int b, uint64_t seed)
{
    using V4 = typename Vec4<MT>::T;
    for (int w = threadIdx.x; w < nc * N; w += blockDim.x) {
        const int sb = w / N, bb = w - sb * N;
        uint32_t x[4] = {(uint32_t)n, (uint32_t)(c0 + sb), (uint32_t)bb, (uint32_t)b};
        philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
        V4 xi;
        xi.x = unit_uniform_t<MT>(x[0]);
        xi.y = unit_uniform_t<MT>(x[1]);
        xi.z = unit_uniform_t<MT>(x[2]);
        xi.w = MT(0);
        sXi[sb * N + bb] = xi;
    }
}

// Barrier over the first nthreads threads (whole warps) of the block with id
// `id`, returning the OR of `v` over them.
__device__ __forceinline__ bool bar_or(int id, int nthreads, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbarrier.cta.red.or.pred po, %2, %3, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// MD substeps of one chain (symplectic Euler), the fluid velocity frozen over
// the LB step.  Each MD thread holds B beads (bead j at slot + j G); L = p.lanes
// consecutive threads share one bead slot.  Each lane owns a list of pair
// tasks of its bead in shared memory -- lane 0 the bond to bead - 1, lane 1
// (lane 0 when L = 1) the bond to bead + 1, then the WCA neighbours it found --
// so the serial part of a substep is about one pair force per bead; the lanes
// sum the force by shuffles and all of them apply the same update (lane 0
// publishes the position).  Velocity, displacement since the start of the step
// and the momentum handed to the fluid stay in registers; positions (start +
// displacement, relative to bead 0's start-of-step position) are
// double-buffered in shared memory as 4-vectors.  One barrier over the MD
// threads per substep -- a warp vote when they fit one warp -- publishes the
// new positions and ORs the flags "some bead left half the Verlet skin" and
// "error".  The noise of a chunk of substeps is drawn up front by every
// thread.  Returns an error code (0 = none); all threads return the same.
template <class MT, int B>
__device__ __forceinline__ int md_substeps(const BeadParams& p, const ChainDev& ch, int N, int64_t n, int b, MT* sXbuf,
                                        MT (*sU)[3], MT (*sV)[3], double (*sR)[3], MT (*sP)[3],
                                        unsigned char (*sNb)[kMaxTasks], int* sErrP)
{
    using V4 = typename Vec4<MT>::T;
    const int tid = threadIdx.x;
    const int maxb = p.max_beads;
    const int L = p.lanes, lshift = __ffs(L) - 1;
    const int nslot = (N + B - 1) / B;
    const int nmd = ((nslot << lshift) + 31) & ~31;  // MD threads: whole warps
    const bool md = tid < nmd;
    const int slot = tid >> lshift, lane = tid & (L - 1);
    const int G = nmd >> lshift;  // slots per bead round
    V4* sX4 = reinterpret_cast<V4*>(sXbuf);  // [2][maxb] positions
    V4* sXi = sX4 + 2 * maxb;                // [chunk][N] noise
    // constants from the chain record (worked out on the host in FP64)
    const MT* mc;
    if constexpr (sizeof(MT) == 8) mc = reinterpret_cast<const MT*>(ch.md_d);
    else mc = reinterpret_cast<const MT*>(ch.md_f);
    const MT dt = mc[kMdDt], dtm = mc[kMdDtm], namp = mc[kMdNamp];
    const MT zeta = mc[kMdZeta];
    const PairConsts<MT> pc{mc[kMdR02], mc[kMdInvR02], mc[kMdKf], mc[kMdSig2], mc[kMdRc2], mc[kMdE24]};
    const bool wca = ch.eps > 0.0;
    const MT rl2 = mc[kMdRl2];  // Verlet radius: WCA cut-off 2^(1/6) sigma + skin
    const MT half_skin2 = mc[kMdHalfSkin2];
    const int cap = kMaxTasks / L;  // task slots of one lane
    int bead[B];
    bool own[B];
    MT X0[B][3], U[B][3], V[B][3], D[B][3], P[B][3], Xref[B][3];
    int bondA[B], bondB[B], nfene[B], ntask[B];
#pragma unroll
    for (int j = 0; j < B; j++) {
        bead[j] = slot + j * G;
        own[j] = md && bead[j] < N;
        const int bj = own[j] ? bead[j] : 0;
        const V4 x0 = sX4[bj];
        X0[j][0] = x0.x;
        X0[j][1] = x0.y;
        X0[j][2] = x0.z;
        for (int a = 0; a < 3; a++) {
            U[j][a] = own[j] ? sU[bj][a] : MT(0);
            V[j][a] = own[j] ? sV[bj][a] : MT(0);
            D[j][a] = P[j][a] = MT(0);
            Xref[j][a] = X0[j][a];
        }
        // bond (FENE) tasks first: lane 0 the bond to bead - 1, lane 1 the
        // bond to bead + 1; a single lane holds both
        bondA[j] = bondB[j] = -1;
        if (own[j]) {
            if (L == 1) {
                if (bj > 0) bondA[j] = bj - 1;
                if (bj + 1 < N) bondB[j] = bj + 1;
            } else if (lane == 0 && bj > 0) {
                bondA[j] = bj - 1;
            } else if (lane == 1 && bj + 1 < N) {
                bondA[j] = bj + 1;
            }
            if (bondA[j] < 0) {
                bondA[j] = bondB[j];
                bondB[j] = -1;
            }
        }
        nfene[j] = (bondA[j] >= 0 ? 1 : 0) + (bondB[j] >= 0 ? 1 : 0);
        ntask[j] = nfene[j];
    }
    MT fext[3];
    for (int a = 0; a < 3; a++) fext[a] = lane == 0 ? (MT)ch.f_ext[a] : MT(0);
    // errors of substep s go to sErrP[s & 1]: a thread that has passed the
    // barrier of substep s can write next only to the other word, so every MD
    // thread reads the same value after that barrier and all stop together
    if (tid < 2) sErrP[tid] = 0;
    __syncthreads();
    auto sync_or = [&](bool v) -> bool {
        if (nmd == 32) {  // one warp: order the shared-memory writes, then vote
            __syncwarp();
            return __any_sync(0xffffffffu, v);
        }
        return bar_or(1, nmd, v);
    };
    bool rebuild = true;  // lists out of date
    const int chunk = namp > MT(0) ? p.noise_chunk : ch.n_md;
    for (int c0 = 0; c0 < ch.n_md; c0 += chunk) {
        const int nc = min(chunk, ch.n_md - c0);
        if (namp > MT(0)) {
            __syncthreads();  // the previous chunk's noise is consumed
            md_noise<MT>(sXi, n, c0, nc, N, b, ch.seed);
            __syncthreads();
        }
        if (md) {
            for (int sb = 0; sb < nc; sb++) {
                const int sub = c0 + sb;
                const V4* Xc = sX4 + (sub & 1) * maxb;
                V4* Xn = sX4 + ((sub + 1) & 1) * maxb;
                bool flag = false;
                MT F[B][3], X[B][3];
#pragma unroll
                for (int j = 0; j < B; j++) {
                    for (int a = 0; a < 3; a++) X[j][a] = X0[j][a] + D[j][a];  // == Xc[bead]
                    if (rebuild && own[j]) {  // lane r scans partners r, r + L, ... after its bonds
                        unsigned char* tasks = &sNb[bead[j]][lane * cap];
                        ntask[j] = 0;
                        if (bondA[j] >= 0) tasks[ntask[j]++] = (unsigned char)bondA[j];
                        if (bondB[j] >= 0) tasks[ntask[j]++] = (unsigned char)bondB[j];
                        int found = 0;
                        if (wca)
                            for (int b2 = lane; b2 < N; b2 += L) {
                                if (b2 == bead[j]) continue;
                                const V4 q = Xc[b2];
                                const MT dx = X[j][0] - q.x, dy = X[j][1] - q.y, dz = X[j][2] - q.z;
                                if (dx * dx + dy * dy + dz * dz < rl2) {
                                    if (ntask[j] < cap) tasks[ntask[j]++] = (unsigned char)b2;
                                    found++;
                                }
                            }
                        if (nfene[j] + found > cap) {  // more neighbours than the list holds
                            sErrP[sub & 1] = LB_ERR_CHAIN;
                            flag = true;
                        }
                        for (int a = 0; a < 3; a++) Xref[j][a] = X[j][a];
                    }
                    // pair forces (pair_force above)
                    for (int a = 0; a < 3; a++) F[j][a] = fext[a];
                    if (own[j]) {
                        const unsigned char* tasks = &sNb[bead[j]][lane * cap];
                        bool bad = false;
                        for (int k = 0; k < ntask[j]; k++)
                            bad |= pair_force<MT>(X[j], Xc[tasks[k]], k < nfene[j], pc, F[j]);
                        if (bad) {
                            sErrP[sub & 1] = LB_ERR_FENE;
                            flag = true;
                        }
                    }
                }
                rebuild = false;
                for (int o = 1; o < L; o <<= 1)  // every lane of an MD warp takes part; xor < L stays in the bead
#pragma unroll
                    for (int j = 0; j < B; j++)
                        for (int a = 0; a < 3; a++) F[j][a] += __shfl_xor_sync(0xffffffffu, F[j][a], o);
#pragma unroll
                for (int j = 0; j < B; j++) {
                    if (!own[j]) continue;
                    const V4 xi = namp > MT(0) ? sXi[sb * N + bead[j]] : V4{};
                    const MT xin[3] = {xi.x, xi.y, xi.z};
                    MT moved = MT(0), xn[3];
                    for (int a = 0; a < 3; a++) {
                        const MT ffric = -zeta * (V[j][a] - U[j][a]);
                        const MT fnoise = namp * xin[a];
                        V[j][a] += dtm * (F[j][a] + ffric + fnoise);
                        D[j][a] += dt * V[j][a];
                        P[j][a] -= (ffric + fnoise) * dt;
                        xn[a] = X0[j][a] + D[j][a];
                        const MT d = xn[a] - Xref[j][a];
                        moved += d * d;
                    }
                    if (lane == 0) {
                        V4 w;
                        w.x = xn[0];
                        w.y = xn[1];
                        w.z = xn[2];
                        w.w = MT(0);
                        Xn[bead[j]] = w;
                    }
                    if (wca && moved > half_skin2) flag = true;
                }
                // publish Xn; any flag: rebuild the lists, or stop on an error
                if (sync_or(flag)) {
                    if (sErrP[sub & 1]) break;
                    rebuild = true;
                }
            }
        }
        __syncthreads();
        if (sErrP[0] || sErrP[1]) break;
    }
    const int err = sErrP[0] ? sErrP[0] : sErrP[1];
    if (err) return err;
#pragma unroll
    for (int j = 0; j < B; j++)
        if (own[j] && lane == 0)
            for (int a = 0; a < 3; a++) {
                sR[bead[j]][a] += (double)D[j][a];
                sV[bead[j]][a] = V[j][a];
                sP[bead[j]][a] = P[j][a];
            }
    __syncthreads();
    return 0;
}

// The same substeps for L = 4 or 8 lanes per bead (one bead per lane group),
// with the update split by component: after the shuffle sum, lane a < 3
// alone advances component a of velocity, displacement and momentum and
// publishes that component of the position; every lane reads its bead's
// position back from shared memory for the pair forces.  The arithmetic of
// each component is that of md_substeps.  The Verlet lists are rebuilt when a
// component of some bead's displacement since the last build exceeds
// (skin / 2) / sqrt(3), which bounds the displacement by skin / 2.
template <class MT, int L>
__device__ __forceinline__ int md_substeps_split(const BeadParams& p, const ChainDev& ch, int N, int64_t n, int b,
                                                 MT* sXbuf, MT (*sU)[3], MT (*sV)[3], double (*sR)[3], MT (*sP)[3],
                                                 unsigned char (*sNb)[kMaxTasks], int* sErrP)
{
    static_assert(L == 4 || L == 8, "component split needs at least three lanes per bead");
    using V4 = typename Vec4<MT>::T;
    constexpr int lshift = L == 8 ? 3 : 2;
    constexpr int cap = kMaxTasks / L;  // task slots of one lane
    const int tid = threadIdx.x;
    const int maxb = p.max_beads;
    const int nmd = ((N << lshift) + 31) & ~31;  // MD threads: whole warps
    const bool md = tid < nmd;
    const int lane = tid & (L - 1);
    const bool own = md && (tid >> lshift) < N;
    const int bead = own ? tid >> lshift : 0;
    const int ca = lane < 3 ? lane : 0;  // component this lane advances
    const bool upd = own && lane < 3;
    V4* sX4 = reinterpret_cast<V4*>(sXbuf);  // [2][maxb] positions, then [chunk][N] noise
    const V4* sXi = sX4 + 2 * maxb;
    const MT* mc;
    if constexpr (sizeof(MT) == 8) mc = reinterpret_cast<const MT*>(ch.md_d);
    else mc = reinterpret_cast<const MT*>(ch.md_f);
    const MT dt = mc[kMdDt], dtm = mc[kMdDtm], namp = mc[kMdNamp], zeta = mc[kMdZeta];
    const PairConsts<MT> pc{mc[kMdR02], mc[kMdInvR02], mc[kMdKf], mc[kMdSig2], mc[kMdRc2], mc[kMdE24]};
    const bool wca = ch.eps > 0.0;
    const MT rl2 = mc[kMdRl2], skin_c2 = mc[kMdSkinComp2];
    // component ca of the bead (lanes >= 3 carry copies they never use)
    const MT x0 = sXbuf[4 * bead + ca];
    const MT u = own ? sU[bead][ca] : MT(0);
    MT v = own ? sV[bead][ca] : MT(0);
    MT d = MT(0), pm = MT(0), dref = MT(0);
    // bond tasks: lane 0 the bond to bead - 1, lane 1 the bond to bead + 1
    int bond = -1;
    if (own && lane == 0 && bead > 0) bond = bead - 1;
    if (own && lane == 1 && bead + 1 < N) bond = bead + 1;
    const int nfene = bond >= 0 ? 1 : 0;
    int ntask = nfene;
    unsigned char* tasks = &sNb[bead][lane * cap];
    MT fext[3];
    for (int a = 0; a < 3; a++) fext[a] = lane == 0 ? (MT)ch.f_ext[a] : MT(0);
    if (tid < 2) sErrP[tid] = 0;
    __syncthreads();
    auto sync_or = [&](bool v) -> bool {
        if (nmd == 32) {
            __syncwarp();
            return __any_sync(0xffffffffu, v);
        }
        return bar_or(1, nmd, v);
    };
    bool rebuild = true;
    const int chunk = namp > MT(0) ? p.noise_chunk : ch.n_md;
    for (int c0 = 0; c0 < ch.n_md; c0 += chunk) {
        const int nc = min(chunk, ch.n_md - c0);
        if (namp > MT(0)) {
            __syncthreads();  // the previous chunk's noise is consumed
            md_noise<MT>(sX4 + 2 * maxb, n, c0, nc, N, b, ch.seed);
            __syncthreads();
        }
        if (md) {
            for (int sb = 0; sb < nc; sb++) {
                const int sub = c0 + sb;
                const V4* Xc = sX4 + (sub & 1) * maxb;
                MT* Xn = sXbuf + 4 * ((sub + 1) & 1) * maxb;
                bool flag = false;
                const V4 xs = Xc[bead];
                const MT X[3] = {xs.x, xs.y, xs.z};
                if (rebuild && own) {  // lane r scans partners r, r + L, ... after its bond
                    ntask = 0;
                    if (bond >= 0) tasks[ntask++] = (unsigned char)bond;
                    int found = 0;
                    if (wca)
                        for (int b2 = lane; b2 < N; b2 += L) {
                            if (b2 == bead) continue;
                            const V4 q = Xc[b2];
                            const MT dx = X[0] - q.x, dy = X[1] - q.y, dz = X[2] - q.z;
                            if (dx * dx + dy * dy + dz * dz < rl2) {
                                if (ntask < cap) tasks[ntask++] = (unsigned char)b2;
                                found++;
                            }
                        }
                    if (nfene + found > cap) {  // more neighbours than the list holds
                        sErrP[sub & 1] = LB_ERR_CHAIN;
                        flag = true;
                    }
                    dref = d;
                }
                rebuild = false;
                MT F[3] = {fext[0], fext[1], fext[2]};
                if (own) {
                    bool bad = false;
                    for (int k = 0; k < ntask; k++) bad |= pair_force<MT>(X, Xc[tasks[k]], k < nfene, pc, F);
                    if (bad) {
                        sErrP[sub & 1] = LB_ERR_FENE;
                        flag = true;
                    }
                }
#pragma unroll
                for (int o = 1; o < L; o <<= 1)  // xor < L stays within the bead's lanes
                    for (int a = 0; a < 3; a++) F[a] += __shfl_xor_sync(0xffffffffu, F[a], o);
                if (upd) {
                    const MT Fa = ca == 0 ? F[0] : (ca == 1 ? F[1] : F[2]);
                    const MT xin = namp > MT(0) ? reinterpret_cast<const MT*>(sXi + sb * N + bead)[ca] : MT(0);
                    const MT ffric = -zeta * (v - u);
                    const MT fnoise = namp * xin;
                    v += dtm * (Fa + ffric + fnoise);
                    d += dt * v;
                    pm -= (ffric + fnoise) * dt;
                    Xn[4 * bead + ca] = x0 + d;
                    const MT dm = d - dref;
                    if (wca && dm * dm > skin_c2) flag = true;
                }
                // publish Xn; any flag: rebuild the lists, or stop on an error
                if (sync_or(flag)) {
                    if (sErrP[sub & 1]) break;
                    rebuild = true;
                }
            }
        }
        __syncthreads();
        if (sErrP[0] || sErrP[1]) break;
    }
    const int err = sErrP[0] ? sErrP[0] : sErrP[1];
    if (err) return err;
    if (upd) {
        sR[bead][ca] += (double)d;
        sV[bead][ca] = v;
        sP[bead][ca] = pm;
    }
    __syncthreads();
    return 0;
}

// Force on a bead at X from a partner at q, added to F where `on` (exactly
// zero otherwise, so that lanes taking different pairs run one instruction
// stream): WCA within the cut-off (the Kremer-Grest chain: WCA acts between
// every pair, bonded or not) plus, for a bond (`fene`), FENE -- the
// expressions of pair_force, the two laws sharing r^2.  Both beads of a pair
// evaluate the same fac from exactly negated differences.  Returns true for a
// bond stretched to R0 or beyond.
template <class MT>
__device__ __forceinline__ bool chain_pair(const MT X[3], const typename Vec4<MT>::T& q, bool fene, bool on,
                                           const PairConsts<MT>& c, bool wca, MT F[3])
{
    const MT rx = X[0] - q.x, ry = X[1] - q.y, rz = X[2] - q.z;
    const MT r2 = rx * rx + ry * ry + rz * rz;
    MT fac = fene ? -c.kf * recip(MT(1) - r2 * c.inv_R02) : MT(0);
    if (wca) {
        const MT inv = recip(r2);
        const MT s2 = c.sig2 * inv, s6 = s2 * s2 * s2;
        fac += r2 < c.rc2 ? c.e24 * (MT(2) * s6 * s6 - s6) * inv : MT(0);
    }
    fac = on ? fac : MT(0);
    F[0] += fac * rx;
    F[1] += fac * ry;
    F[2] += fac * rz;
    return on && fene && r2 >= c.R02;
}

// Verlet list of bead g (pairs at least three apart within sqrt(rl2)) from
// the positions X, written to lst by the two lanes of the bead: each scans
// alternate partners, a count pass, then each writes its finds after the
// other's.  Kept out of line so that the substep loop stays small in the
// instruction cache; called by every lane of the warp.  Returns the length
// (entries past kMaxTasks are not written).
template <class MT>
__device__ __noinline__ int rebuild_chain_list(const typename Vec4<MT>::T* X, unsigned char* lst, int g, int role, int N,
                                               bool own, MT rl2)
{
    using V4 = typename Vec4<MT>::T;
    const V4 xb = X[own ? g : 0];
    int cnt = 0;
    if (own)
        for (int p2 = role; p2 < N; p2 += 2) {
            const int dd = p2 - g;
            if (dd >= -2 && dd <= 2) continue;
            const V4 q = X[p2];
            const MT dx = xb.x - q.x, dy = xb.y - q.y, dz = xb.z - q.z;
            cnt += dx * dx + dy * dy + dz * dz < rl2;
        }
    const int c_other = __shfl_xor_sync(0xffffffffu, cnt, 1);
    int k = role ? c_other : 0;
    if (own)
        for (int p2 = role; p2 < N; p2 += 2) {
            const int dd = p2 - g;
            if (dd >= -2 && dd <= 2) continue;
            const V4 q = X[p2];
            const MT dx = xb.x - q.x, dy = xb.y - q.y, dz = xb.z - q.z;
            if (dx * dx + dy * dy + dz * dz < rl2) {
                if (k < kMaxTasks) lst[k] = (unsigned char)p2;
                k++;
            }
        }
    return own ? cnt + c_other : 0;
}

// The MD substeps with two lanes per bead in chain order: thread t holds
// bead t / 2 in role t & 1.  Each lane reads two partners from the positions
// published in shared memory -- role 0 the bonded neighbours (FENE + WCA),
// role 1 the beads two apart (WCA) -- and the pairs at least three apart come
// from Verlet lists split between the two lanes (role r takes entries r,
// r + 2, ...; the first two of a lane as bytes of one register).  The lanes
// of a bead sum their forces with one shuffle and apply the same update, so
// both hold the bead's state; role 0 publishes the position.  Every branch of
// the force phase is uniform over the warp (pair slots are masked, not
// skipped), so a lane's pair computations interleave.  One barrier over the
// MD threads per substep publishes the positions and ORs the flags "some bead
// left half the Verlet skin" and "error" (a warp vote when the chain fits one
// warp).  The lists are built by the whole block before the substeps from the
// start positions and rebuilt by the MD threads after a flagged barrier.
// Symplectic Euler as in md_substeps.  Called by every thread of the block;
// returns an error code (0 = none), the same in all threads.
template <class MT>
__device__ __forceinline__ int md_chain_pairs(const BeadParams& p, const ChainDev& ch, int N, int64_t n, int b,
                                              MT* sXbuf, MT (*sU)[3], MT (*sV)[3], double (*sR)[3], MT (*sP)[3],
                                              unsigned char (*sNb)[kMaxTasks], int* sErrP)
{
    using V4 = typename Vec4<MT>::T;
    __shared__ int sNbN[kMaxBeads];  // listed partners of each bead
    __shared__ int sErrB;            // list overflow of the block's build
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int maxb = p.max_beads;
    V4* sX4 = reinterpret_cast<V4*>(sXbuf);  // [2][maxb] positions, then [chunk][N] noise
    const V4* sXi = sX4 + 2 * maxb;
    const MT* mc;
    if constexpr (sizeof(MT) == 8) mc = reinterpret_cast<const MT*>(ch.md_d);
    else mc = reinterpret_cast<const MT*>(ch.md_f);
    const MT dt = mc[kMdDt], dtm = mc[kMdDtm], namp = mc[kMdNamp], zeta = mc[kMdZeta];
    const PairConsts<MT> pc{mc[kMdR02], mc[kMdInvR02], mc[kMdKf], mc[kMdSig2], mc[kMdRc2], mc[kMdE24]};
    const bool wca = ch.eps > 0.0;
    const MT rl2 = mc[kMdRl2], half_skin2 = mc[kMdHalfSkin2];
    // errors of substep s go to sErrP[s & 1]: a thread that has passed the
    // barrier of substep s can write next only to the other word, so every MD
    // thread reads the same value after that barrier and all stop together
    if (tid < 2) sErrP[tid] = 0;
    if (tid == 0) sErrB = 0;
    __syncthreads();
    // Verlet lists of the pairs at least three apart, from the start positions
    // (buffer 0): eight threads per bead scan every eighth partner and merge
    // their finds in order by a prefix sum over the eight
    if (wca) {
        for (int base = 0; base < 8 * N; base += nthr) {
            const int e = base + tid;
            const bool act = e < 8 * N;
            const int bb = act ? e >> 3 : 0, r = e & 7;
            uint32_t m = 0;  // bit k: partner r + 8 k (N <= 256)
            if (act) {
                const V4 xb = sX4[bb];
                for (int k = 0, p2 = r; p2 < N; k++, p2 += 8) {
                    const int dd = p2 - bb;
                    if (dd >= -2 && dd <= 2) continue;
                    const V4 q = sX4[p2];
                    const MT dx = xb.x - q.x, dy = xb.y - q.y, dz = xb.z - q.z;
                    if (dx * dx + dy * dy + dz * dz < rl2) m |= 1u << k;
                }
            }
            const int cnt = __popc(m);
            int incl = cnt;
            for (int o = 1; o < 8; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o, 8);
                if (r >= o) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 7, 8);
            if (act) {
                int k = incl - cnt;
                for (uint32_t mm = m; mm; mm &= mm - 1, k++)
                    if (k < kMaxTasks) sNb[bb][k] = (unsigned char)(r + 8 * (__ffs(mm) - 1));
                if (r == 7) {
                    sNbN[bb] = total;
                    if (total > kMaxTasks) sErrB = LB_ERR_CHAIN;  // more neighbours than the list holds
                }
            }
        }
    }
    __syncthreads();
    if (sErrB) return sErrB;

    const int nmd = (2 * N + 31) & ~31;  // MD threads: whole warps
    const bool md = tid < nmd;
    const int g = tid >> 1, role = tid & 1;
    const bool own = md && g < N;
    const int gg = own ? g : 0;
    const V4 xs = sX4[gg];
    const MT x0[3] = {own ? xs.x : MT(0), own ? xs.y : MT(0), own ? xs.z : MT(0)};
    MT u[3], v[3], d[3] = {MT(0), MT(0), MT(0)}, pm[3] = {MT(0), MT(0), MT(0)}, dref[3] = {MT(0), MT(0), MT(0)};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        u[a] = own ? sU[gg][a] : MT(0);
        v[a] = own ? sV[gg][a] : MT(0);
    }
    // the two fixed partners of this lane: g -/+ 1 (role 0) or g -/+ 2 (role 1)
    const int off = role ? 2 : 1;
    const bool onl = own && g - off >= 0, onr = own && g + off < N;
    const int il = onl ? g - off : gg, ir = onr ? g + off : gg;
    const bool fene = role == 0;
    MT fx[3];
    for (int a = 0; a < 3; a++) fx[a] = role == 0 ? (MT)ch.f_ext[a] : MT(0);  // added once per bead
    // this lane's share of the list: entries role, role + 2, ...; the first
    // two as bytes of li (unused slots name the bead itself: a valid
    // position, masked out), and the warp's largest share
    int nl = own && wca ? sNbN[gg] : 0;
    uint32_t li = 0;
    int mine = 0, kmax = 0;
    auto pack = [&]() {
        mine = nl > role ? (nl - role + 1) >> 1 : 0;
        li = 0;
#pragma unroll
        for (int s = 0; s < 2; s++) li |= (uint32_t)(s < mine ? sNb[gg][role + 2 * s] : gg) << (8 * s);  // < kMaxTasks
        kmax = __reduce_max_sync(0xffffffffu, mine);
    };
    if (md) pack();
    auto sync_or = [&](bool f) -> bool {
        if (nmd == 32) {
            __syncwarp();
            return __any_sync(0xffffffffu, f);
        }
        return bar_or(1, nmd, f);
    };
    const int chunk = namp > MT(0) ? p.noise_chunk : ch.n_md;
    for (int c0 = 0; c0 < ch.n_md; c0 += chunk) {
        const int nc = min(chunk, ch.n_md - c0);
        if (namp > MT(0)) {
            __syncthreads();  // the previous chunk's noise is consumed
            md_noise<MT>(sX4 + 2 * maxb, n, c0, nc, N, b, ch.seed);
            __syncthreads();
        }
        if (md) {
            for (int sb = 0; sb < nc; sb++) {
                const int sub = c0 + sb;
                const V4* Xc = sX4 + (sub & 1) * maxb;
                V4* Xn = sX4 + ((sub + 1) & 1) * maxb;
                // the lane's two fixed partners and its first two list slots
                // in one branch-free block, so that the four pair
                // computations interleave (empty slots are masked)
                const V4 xi = namp > MT(0) ? sXi[sb * N + gg] : V4{};
                const V4 ql = Xc[il], qr = Xc[ir], q0 = Xc[li & 255u], q1 = Xc[(li >> 8) & 255u];
                const MT X[3] = {x0[0] + d[0], x0[1] + d[1], x0[2] + d[2]};
                MT F[3] = {fx[0], fx[1], fx[2]}, G[3] = {MT(0), MT(0), MT(0)};
                bool stretched = chain_pair<MT>(X, ql, fene, onl, pc, wca, F);
                stretched |= chain_pair<MT>(X, qr, fene, onr, pc, wca, G);
                chain_pair<MT>(X, q0, false, wca && 0 < mine, pc, wca, F);
                chain_pair<MT>(X, q1, false, wca && 1 < mine, pc, wca, G);
#pragma unroll
                for (int a = 0; a < 3; a++) F[a] += G[a];
                // the rest of the list (rare: a bead with more than four
                // listed partners), one slot per trip, read from shared memory
                for (int s = 2; s < kmax; s++) {
                    const int k = role + 2 * s;
                    const bool on = s < mine && k < kMaxTasks;  // an overflowing list stops at the next barrier
                    chain_pair<MT>(X, Xc[on ? sNb[gg][k] : gg], false, on, pc, true, F);
                }
#pragma unroll
                for (int a = 0; a < 3; a++) F[a] += __shfl_xor_sync(0xffffffffu, F[a], 1);
                const MT xin[3] = {xi.x, xi.y, xi.z};
                MT m2 = MT(0), xn[3];
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const MT ffric = -zeta * (v[a] - u[a]);
                    const MT fnoise = namp * xin[a];
                    v[a] += dtm * (F[a] + ffric + fnoise);
                    d[a] += dt * v[a];
                    pm[a] -= (ffric + fnoise) * dt;
                    xn[a] = x0[a] + d[a];
                    const MT dm = d[a] - dref[a];
                    m2 += dm * dm;
                }
                if (own && role == 0) {
                    V4 w;
                    w.x = xn[0];
                    w.y = xn[1];
                    w.z = xn[2];
                    w.w = MT(0);
                    Xn[g] = w;
                }
                if (stretched) sErrP[sub & 1] = LB_ERR_FENE;
                const bool moved = own && wca && m2 > half_skin2;
                // publish Xn; any flag: stop on an error, or rebuild the lists
                if (sync_or(stretched || moved)) {
                    if (sErrP[sub & 1]) break;
                    nl = rebuild_chain_list<MT>(Xn, sNb[gg], g, role, N, own, rl2);
                    // more neighbours than the list holds: the error stops
                    // the next barrier (or the chunk's)
                    if (nl > kMaxTasks) sErrP[(sub + 1) & 1] = LB_ERR_CHAIN;
#pragma unroll
                    for (int a = 0; a < 3; a++) dref[a] = d[a];
                    __syncwarp();  // both lanes' finds are in place
                    pack();
                }
            }
        }
        __syncthreads();
        if (sErrP[0] || sErrP[1]) break;
    }
    const int err = sErrP[0] ? sErrP[0] : sErrP[1];
    if (err) return err;
    if (own && role == 0)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            sR[g][a] += (double)d[a];
            sV[g][a] = v[a];
            sP[g][a] = pm[a];
        }
    __syncthreads();
    return 0;
}

template <int ST>
__global__ void __launch_bounds__(kBeadThreadsMax) k_bead_couple(BeadParams p)
{
    using S = Stor<ST>;
    using A = typename S::A;
    using MT = typename std::conditional<ST == kF64, double, float>::type;
    const int tid = threadIdx.x, nthr = blockDim.x;
    // The chain and box records, the status and the step number are read once
    // into shared memory: later phases would otherwise reload them from L2
    // (the gather evicts L1) while the stream-collide launch keeps the memory
    // system busy, and one reading of the status serves the whole block
    // (another launch may set it meanwhile).
    __shared__ ChainDev sCh;
    __shared__ BoxDev sBd;
    __shared__ int sGo;
    __shared__ int64_t sStep;
    {
        const int b0 = p.chains[blockIdx.x].box;
        static_assert(sizeof(ChainDev) % 8 == 0 && sizeof(BoxDev) % 8 == 0, "records copied in 8-byte words");
        constexpr int wc = (int)(sizeof(ChainDev) / 8), wb = (int)(sizeof(BoxDev) / 8);
        for (int w = tid; w < wc + wb; w += nthr) {
            if (w < wc)
                reinterpret_cast<uint64_t*>(&sCh)[w] = reinterpret_cast<const uint64_t*>(p.chains + blockIdx.x)[w];
            else
                reinterpret_cast<uint64_t*>(&sBd)[w - wc] = reinterpret_cast<const uint64_t*>(p.boxes + b0)[w - wc];
        }
        if (tid == nthr - 1) sGo = p.status[b0] == 0;
        if (tid == nthr - 2) sStep = *p.step;
    }
    __syncthreads();
    const ChainDev& ch = sCh;
    const BoxDev& bd = sBd;
    const int N = ch.nbeads;
    const int b = ch.box;
    if (N <= 0 || !sGo) return;
    const int Ei = bd.E, per = bd.per_mask;
    const int64_t n3 = bd.n3;
    const int64_t n = sStep;

    __shared__ double sR[kMaxBeads][3];      // start-of-step, then end-of-step positions
    __shared__ MT sD[kMaxBeads][3];          // start-of-step offsets inside the stencil cell
    __shared__ int sBase[kMaxBeads][3];      // start-of-step stencil corner
    __shared__ MT sU[kMaxBeads][3];          // fluid velocity at each bead
    __shared__ MT sV[kMaxBeads][3];          // velocities
    __shared__ MT sP[kMaxBeads][3];          // momentum given to the fluid
    __shared__ unsigned char sNb[kMaxBeads][kMaxTasks];
    __shared__ unsigned char sSt[kMaxBeads][kMaxStencilNb];  // beads whose stencil may share a site
    __shared__ int sStN[kMaxBeads];
    __shared__ double sRc[3];
    __shared__ A sAcc[3];  // body acceleration in the collision type
    __shared__ MT sRed[2][kBeadThreadsMax / 32][3];
    __shared__ int sErr;
    extern __shared__ __align__(32) unsigned char bead_dyn[];
    MT* sXbuf = reinterpret_cast<MT*>(bead_dyn);       // [2][max_beads] 4-vectors, then the noise

    double* pos = p.pos + 3 * ch.bead_off;
    double* vel = p.vel + 3 * ch.bead_off;
    if (tid == 0) {
        sErr = 0;
        double acc[3];  // body acceleration of step n, also handed to the forced sites
        frame_accel_at(bd, p.faccel, p.ring_slots, n, acc);
        for (int a = 0; a < 3; a++) {
            sRc[a] = pos[a];
            sAcc[a] = (A)acc[a];
            p.chain_accel[4 * blockIdx.x + a] = acc[a];
        }
    }
    __syncthreads();

    // 1. stencil of the start-of-step position (one thread per bead)
    for (int bb = tid; bb < N; bb += nthr) {
        for (int a = 0; a < 3; a++) {
            const double R = pos[3 * bb + a];
            sR[bb][a] = R;
            sV[bb][a] = (MT)vel[3 * bb + a];
            const double fl = floor(R);
            sD[bb][a] = (MT)(R - fl);
            long long i0 = (long long)fl;
            if (!((per >> a) & 1)) {
                if (i0 < 1 || i0 + 1 > Ei - 2) sErr = LB_ERR_BEAD_OOB;
                sBase[bb][a] = (int)i0;
            } else {
                sBase[bb][a] = (int)(((i0 % Ei) + Ei) % Ei);
            }
            sXbuf[4 * bb + a] = (MT)(R - sRc[a]);  // 4-vector layout of the MD phase
        }
    }
    __syncthreads();
    if (sErr) {
        if (tid == 0) set_status(&p.status[b], sErr);
        return;
    }
    // trilinear weight of corner c of bead bb (MT precision: FP32 on the reduced paths)
    auto weight = [&](int bb, int c) -> MT {
        const MT d0 = sD[bb][0], d1 = sD[bb][1], d2 = sD[bb][2];
        return ((c & 1) ? d0 : MT(1) - d0) * ((c & 2) ? d1 : MT(1) - d1) * ((c & 4) ? d2 : MT(1) - d2);
    };

    // 2. fluid velocity at the beads: eight threads per bead, one corner each
    const typename S::E* Ab = reinterpret_cast<const typename S::E*>(p.A) + bd.f_off;
    for (int base = 0; base < 8 * N; base += nthr) {
        const int e = base + tid;
        const bool act = e < 8 * N;
        MT uc[3] = {0, 0, 0};
        if (act) {
            const int bb = e >> 3, c = e & 7;
            int s[3] = {sBase[bb][0] + (c & 1), sBase[bb][1] + ((c >> 1) & 1), sBase[bb][2] + ((c >> 2) & 1)};
            for (int a = 0; a < 3; a++)
                if ((per >> a) & 1) s[a] = wrapi(s[a], Ei);
            A f[kQ], dr, j[3];
            pull_site<ST>(Ab, n3, Ei, per, s[0], s[1], s[2], f);
            moments<A>(f, dr, j);
            const A rho = A(1) + dr;
            const MT w8 = weight(bb, c);
            for (int a = 0; a < 3; a++) uc[a] = w8 * (MT)((j[a] + A(0.5) * rho * sAcc[a]) / rho);
        }
        for (int a = 0; a < 3; a++) {
            uc[a] += __shfl_xor_sync(0xffffffffu, uc[a], 1);
            uc[a] += __shfl_xor_sync(0xffffffffu, uc[a], 2);
            uc[a] += __shfl_xor_sync(0xffffffffu, uc[a], 4);
        }
        if (act && (e & 7) == 0)
            for (int a = 0; a < 3; a++) sU[e >> 3][a] = (MT)uc[a];
    }
    __syncthreads();

    // 3. MD substeps (md_substeps below)
    {
        __shared__ int sErrP[2];
        int err;
        if (p.beads_per_thread == 0)
            err = md_chain_pairs<MT>(p, ch, N, n, b, sXbuf, sU, sV, sR, sP, sNb, sErrP);
        else if (p.beads_per_thread == 1 && p.lanes == 8)
            err = md_substeps_split<MT, 8>(p, ch, N, n, b, sXbuf, sU, sV, sR, sP, sNb, sErrP);
        else if (p.beads_per_thread == 1 && p.lanes == 4)
            err = md_substeps_split<MT, 4>(p, ch, N, n, b, sXbuf, sU, sV, sR, sP, sNb, sErrP);
        else if (p.beads_per_thread == 2)
            err = md_substeps<MT, 2>(p, ch, N, n, b, sXbuf, sU, sV, sR, sP, sNb, sErrP);
        else
            err = md_substeps<MT, 1>(p, ch, N, n, b, sXbuf, sU, sV, sR, sP, sNb, sErrP);
        if (err) {
            if (tid == 0) set_status(&p.status[b], err);
            return;
        }
    }

    // 4. centre of mass pinned at the box centre (one thread per bead; only
    //    the warps holding beads reduce).  The sums run in MT over the offsets
    //    from bead 0's start-of-step position, which are small: FP64 is slow
    //    on this part, and the pin is re-applied every step, so the FP32
    //    rounding of one step's shift does not accumulate.
    double R[3] = {0, 0, 0};
    MT V[3] = {0, 0, 0};
    if (tid < N)
        for (int a = 0; a < 3; a++) {
            R[a] = sR[tid][a];
            V[a] = sV[tid][a];
        }
    if (ch.pin_com >= 1) {
        const int warp = tid >> 5, lane = tid & 31, nbw = (N + 31) >> 5;
        if (warp < nbw)
            for (int pass = 0; pass < 2; pass++) {
                MT s[3];
                for (int a = 0; a < 3; a++) {
                    s[a] = tid < N ? (pass == 0 ? (MT)(R[a] - sRc[a]) : V[a]) : MT(0);
                    for (int o = 16; o > 0; o >>= 1) s[a] += __shfl_xor_sync(0xffffffffu, s[a], o);
                }
                if (lane == 0)
                    for (int a = 0; a < 3; a++) sRed[pass][warp][a] = s[a];
            }
        __syncthreads();
        if (tid < N) {
            MT com[3] = {0, 0, 0}, vcm[3] = {0, 0, 0};
            for (int w = 0; w < nbw; w++)
                for (int a = 0; a < 3; a++) {
                    com[a] += sRed[0][w][a];
                    vcm[a] += sRed[1][w][a];
                }
            const double centre = 0.5 * (Ei - 1);
            const MT inv_n = sizeof(MT) == 8 ? (MT)ch.md_d[kMdInvN] : (MT)ch.md_f[kMdInvN];
            for (int a = 0; a < 3; a++) {
                R[a] += (centre - sRc[a]) - (double)(com[a] * inv_n);
                if (ch.pin_com >= 2) V[a] = V[a] - vcm[a] * inv_n;
            }
        }
    }
    if (tid < N)
        for (int a = 0; a < 3; a++) {
            pos[3 * tid + a] = R[a];
            vel[3 * tid + a] = (double)V[a];
        }
    if (p.hist_slots > 0 && tid < N) {  // the trajectory ring: positions after step n + 1
        double* h = p.hist + ((n + 1) % p.hist_slots) * p.hist_stride + 3 * (int64_t)ch.bead_off;
        for (int a = 0; a < 3; a++) h[3 * tid + a] = R[a];
    }

    // 5. force density at the stencil sites: every entry sums, in bead order,
    //    the contributions of all beads whose stencil holds its site; entries
    //    whose site an earlier bead already holds are marked duplicates.
    //    Only beads whose stencil corner lies within one cell of this bead's on
    //    every axis can share a site: each bead first lists those (in bead
    //    order, itself included), then each entry scans its bead's list only.
    ForceEntry* fl = p.forces + ch.force_off;
    //    Eight threads per bead scan consecutive eighths of the chain and
    //    merge their finds in order by a prefix sum over the eight.
    {
        const int part = (N + 7) >> 3;  // <= 32 beads per thread
        for (int base = 0; base < 8 * N; base += nthr) {
            const int e = base + tid;
            const bool act = e < 8 * N;
            const int bb = act ? e >> 3 : 0, r = e & 7;
            const int lo = r * part, hi = min(N, lo + part);
            uint32_t m = 0;
            if (act)
                for (int b2 = lo; b2 < hi; b2++) {
                    bool near = true;
                    for (int a = 0; a < 3; a++) {
                        int d = sBase[b2][a] - sBase[bb][a];
                        if ((per >> a) & 1) {
                            d = wrapi(d, Ei);
                            if (d > Ei / 2) d -= Ei;
                        }
                        near = near && d >= -1 && d <= 1;
                    }
                    if (near) m |= 1u << (b2 - lo);
                }
            const int cnt = __popc(m);
            int incl = cnt;
            for (int o = 1; o < 8; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o, 8);
                if (r >= o) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 7, 8);
            if (act) {
                int k = incl - cnt;
                for (uint32_t mm = m; mm; mm &= mm - 1, k++)
                    if (k < kMaxStencilNb) sSt[bb][k] = (unsigned char)(lo + __ffs(mm) - 1);
                if (r == 7) sStN[bb] = total <= kMaxStencilNb ? total : -1;  // -1: too many, scan every bead
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < 8 * N; e += nthr) {
        const int bb = e >> 3, c = e & 7;
        int s[3] = {sBase[bb][0] + (c & 1), sBase[bb][1] + ((c >> 1) & 1), sBase[bb][2] + ((c >> 2) & 1)};
        for (int a = 0; a < 3; a++)
            if ((per >> a) & 1) s[a] = wrapi(s[a], Ei);
        MT g[3] = {0, 0, 0};
        bool dup = false;
        const int nlist = sStN[bb];
        const int nscan = nlist >= 0 ? nlist : N;
        for (int k = 0; k < nscan; k++) {
            const int b2 = nlist >= 0 ? (int)sSt[bb][k] : k;
            int o[3];
            bool in = true;
            for (int a = 0; a < 3; a++) {
                int d = s[a] - sBase[b2][a];
                if ((per >> a) & 1) d = wrapi(d, Ei);
                o[a] = d;
                in = in && (d == 0 || d == 1);
            }
            if (!in) continue;
            if (b2 < bb) dup = true;
            const MT w8 = weight(b2, o[0] + 2 * o[1] + 4 * o[2]);
            for (int a = 0; a < 3; a++) g[a] += w8 * sP[b2][a];
        }
        ForceEntry fe;
        fe.site = dup ? -1 : (int32_t)(((int64_t)s[2] * Ei + s[1]) * Ei + s[0]);
        fe.pad = 0;
        for (int a = 0; a < 3; a++) fe.g[a] = (double)g[a];
        fl[e] = fe;
    }
}

// ---------------------------------------------------------------------------
// Forced re-collision: the sites that carry a bead force density g are
// collided again with rho a + g (Guo forcing) and overwrite B.  Block 0
// advances the device step counter once all of its own work is done.
// ---------------------------------------------------------------------------
template <int ST>
__global__ void __launch_bounds__(kForcedThreads) k_forced(ForcedParams p)
{
    // the next step's stream-collide (a programmatic dependent) may be
    // scheduled now; it waits on the device for this kernel to complete
    asm volatile("griddepcontrol.launch_dependents;");
    // this kernel is itself a programmatic dependent of the stream-collide
    // before it: wait for that grid to complete and its stores to be visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    using S = Stor<ST>;
    using A = typename S::A;
    const int chain = (int)blockIdx.x / p.splits, part = (int)blockIdx.x - chain * p.splits;
    if (chain < p.nchains) {
        const ChainDev& ch = p.chains[chain];
        const int b = ch.box, nb = ch.nbeads;
        const ForceEntry* fl = p.forces + ch.force_off;
        // the entry, the status and the box record are independent loads:
        // issue them together (e stays inside the chain's entries)
        for (int e = part * blockDim.x + threadIdx.x; e < 8 * nb; e += p.splits * blockDim.x) {
            const ForceEntry fe = fl[e];
            const int st = p.status[b];
            const BoxDev& bd = p.boxes[b];
            const int Ei = bd.E, per = bd.per_mask;
            const int64_t n3 = bd.n3;
            const typename S::E* Ab = reinterpret_cast<const typename S::E*>(p.A) + bd.f_off;
            typename S::E* Bb = reinterpret_cast<typename S::E*>(p.B) + bd.f_off;
            if (fe.site < 0 || st != 0) continue;
            const int x = fe.site % Ei, y = (fe.site / Ei) % Ei, z = fe.site / (Ei * Ei);
            A f[kQ], dr, j[3];
            pull_site<ST>(Ab, n3, Ei, per, x, y, z, f);
            moments<A>(f, dr, j);
            const A rho = A(1) + dr;
            A F[3], u[3];
            for (int a = 0; a < 3; a++) {
                F[a] = rho * (A)p.chain_accel[4 * chain + a] + (A)fe.g[a];
                u[a] = (j[a] + A(0.5) * F[a]) / rho;
            }
            const A om = A(1) / (A)bd.tau;
            const A usq = A(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            const A uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
#pragma unroll
            for (int i = 0; i < kQ; i++) {
                const A w = wgt<A>(i);
                const A cu = cvec(i, 0) * u[0] + cvec(i, 1) * u[1] + cvec(i, 2) * u[2];
                const A cF = cvec(i, 0) * F[0] + cvec(i, 1) * F[1] + cvec(i, 2) * F[2];
                const A deq = w * (dr + rho * (A(3) * cu + A(4.5) * cu * cu - usq));
                A val = f[i] + om * (deq - f[i]);
                val += (A(1) - A(0.5) * om) * w * (A(3) * (cF - uF) + A(9) * cu * cF);
                Bb[(int64_t)i * n3 + fe.site] = S::out(val);
            }
        }
    }
    if (blockIdx.x == 0) {
        __syncthreads();
        if (threadIdx.x == 0) {
            *p.step += 1;
            *p.tile_counter = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Initial condition: equilibrium with rho = 1 and velocity u0 on every site.
// ---------------------------------------------------------------------------
// u0 lives on the coarse grid [3][Ec^3] (the sites themselves when z = 1); with
// z > 1 a site takes the trilinear interpolation of its eight coarse
// neighbours (Sec. 2: the initial field interpolated linearly).
template <int ST>
__global__ void k_init(typename Stor<ST>::E* Ab, BoxDev bd, const typename Stor<ST>::R* u0)
{
    using S = Stor<ST>;
    using A = typename S::A;
    using R = typename S::R;
    const int64_t n3 = bd.n3, c3 = (int64_t)bd.Ec * bd.Ec * bd.Ec;
    const int Ei = bd.E, z = bd.zoom, Ec = bd.Ec;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n3; s += (int64_t)gridDim.x * blockDim.x) {
        A u[3];
        if (z == 1) {
            for (int c = 0; c < 3; c++) u[c] = (A)u0[c * c3 + s];
        } else {
            const int xyz[3] = {(int)(s % Ei), (int)((s / Ei) % Ei), (int)(s / ((int64_t)Ei * Ei))};
            int i0[3], i1[3];
            R fr[3];
            for (int a = 0; a < 3; a++) {
                i0[a] = xyz[a] / z;
                i1[a] = i0[a] + 1 < Ec ? i0[a] + 1 : i0[a];
                fr[a] = (R)(xyz[a] - i0[a] * z) / (R)z;
            }
            for (int c = 0; c < 3; c++) {
                R acc = R(0);
                for (int k = 0; k < 8; k++) {
                    const int X = (k & 1) ? i1[0] : i0[0], Y = (k & 2) ? i1[1] : i0[1], Z = (k & 4) ? i1[2] : i0[2];
                    const R w = ((k & 1) ? fr[0] : R(1) - fr[0]) * ((k & 2) ? fr[1] : R(1) - fr[1]) *
                                ((k & 4) ? fr[2] : R(1) - fr[2]);
                    acc += w * u0[c * c3 + ((int64_t)Z * Ec + Y) * Ec + X];
                }
                u[c] = (A)acc;
            }
        }
        const A usq = A(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
        for (int i = 0; i < kQ; i++) {
            const A cu = cvec(i, 0) * u[0] + cvec(i, 1) * u[1] + cvec(i, 2) * u[2];
            Ab[(int64_t)i * n3 + s] = S::out(wgt<A>(i) * (A(3) * cu + A(4.5) * cu * cu - usq));
        }
    }
}

// ---------------------------------------------------------------------------
// Observables: density and velocity (what = 0: rho, 1: u) and raw deviations.
// ---------------------------------------------------------------------------
template <int ST>
__global__ void k_fields(const typename Stor<ST>::E* Ab, BoxDev bd, int what, typename Stor<ST>::R* dst)
{
    using S = Stor<ST>;
    using A = typename S::A;
    const int Ei = bd.E, per = bd.per_mask;
    const int64_t n3 = bd.n3;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n3; s += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % Ei), y = (int)((s / Ei) % Ei), z = (int)(s / ((int64_t)Ei * Ei));
        const bool bnd = (!(per & 1) && (x == 0 || x == Ei - 1)) || (!(per & 2) && (y == 0 || y == Ei - 1)) ||
                         (!(per & 4) && (z == 0 || z == Ei - 1));
        A f[kQ], dr, j[3];
        if (bnd) {
            for (int i = 0; i < kQ; i++) f[i] = S::in(Ab[(int64_t)i * n3 + s]);
        } else {
            pull_site<ST>(Ab, n3, Ei, per, x, y, z, f);
        }
        moments<A>(f, dr, j);
        const A rho = A(1) + dr;
        if (what == 0) {
            dst[s] = (typename S::R)rho;
        } else {
            for (int a = 0; a < 3; a++) {
                const A ja = bnd ? j[a] : j[a] + A(0.5) * rho * (A)bd.accel[a];
                dst[(int64_t)a * n3 + s] = (typename S::R)(ja / rho);
            }
        }
    }
}

template <int ST>
__global__ void k_read_dev(const typename Stor<ST>::E* Ab, int64_t count, typename Stor<ST>::R* dst)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < count; s += (int64_t)gridDim.x * blockDim.x)
        dst[s] = (typename Stor<ST>::R)Stor<ST>::in(Ab[s]);
}

// ---------------------------------------------------------------------------
// Conservation sums in FP64: block (chunk, box) sums its sites into a partial,
// then one thread per box adds the partials in chunk order.
// ---------------------------------------------------------------------------
constexpr int kConsThreads = 256;
constexpr int kConsSitesPerThread = 16;
constexpr int64_t kConsChunk = (int64_t)kConsThreads * kConsSitesPerThread;

template <int ST>
__global__ void __launch_bounds__(kConsThreads) k_cons_partial(const void* Araw, const BoxDev* boxes, int64_t chunks,
                                                               double* partial)
{
    using S = Stor<ST>;
    const int b = blockIdx.y;
    const BoxDev& bd = boxes[b];
    const int64_t n3 = bd.n3;
    const int64_t c0 = (int64_t)blockIdx.x * kConsChunk;
    if (c0 >= n3) return;
    const typename S::E* Ab = reinterpret_cast<const typename S::E*>(Araw) + bd.f_off;
    double acc[4] = {0, 0, 0, 0};
    for (int k = 0; k < kConsSitesPerThread; k++) {
        const int64_t s = c0 + (int64_t)k * kConsThreads + threadIdx.x;
        if (s >= n3) break;
#pragma unroll
        for (int i = 0; i < kQ; i++) {
            const double d = (double)S::in(Ab[(int64_t)i * n3 + s]);
            acc[0] += d;
            if (cvec(i, 0)) acc[1] += cvec(i, 0) * d;
            if (cvec(i, 1)) acc[2] += cvec(i, 1) * d;
            if (cvec(i, 2)) acc[3] += cvec(i, 2) * d;
        }
    }
    __shared__ double red[kConsThreads / 32][4];
    for (int a = 0; a < 4; a++)
        for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 4; a++) red[threadIdx.x >> 5][a] = acc[a];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0, 0, 0, 0};
        for (int w = 0; w < kConsThreads / 32; w++)
            for (int a = 0; a < 4; a++) t[a] += red[w][a];
        for (int a = 0; a < 4; a++) partial[((int64_t)b * chunks + blockIdx.x) * 4 + a] = t[a];
    }
}

__global__ void k_cons_final(const BoxDev* boxes, const ChainDev* chains, int nboxes, int64_t chunks,
                             const double* partial, const double* vel, double* out, int32_t* status);

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
template <int ST>
constexpr int kVW = ST == kF64 ? 2 : (ST == kF32 ? 4 : 8);

inline int grid_for(int64_t n, int threads, int cap = 152 * 16)
{
    int64_t g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

template <int ST, int SPT, int KIND>
cudaError_t launch_staged(const SCParams& p, int ctas, cudaStream_t s)
{
    using G = Staged<ST, SPT>;
    static int attr_done[kMaxDevices] = {};  // per instantiation and device
    cudaError_t e = smem_attr_per_device(k_stream_collide_staged<ST, SPT, KIND>, G::kSmemBytes, attr_done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if (ctas <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    int64_t grid = ctas > 0 ? ctas : sms;
    if (grid > p.total_tiles) grid = p.total_tiles;
    if (grid < 1) return cudaSuccess;
    // programmatic dependent launch: the blocks may be scheduled before the
    // previous kernel on the stream completes (they wait for it on the device)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kStagedThreads);
    cfg.dynamicSmemBytes = G::kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_stream_collide_staged<ST, SPT, KIND>, p);
}

template <int ST>
cudaError_t Launch<ST>::stream_collide(const SCParams& p, int kernel, int threads, int ctas, int vw, cudaStream_t s)
{
    if (kernel == LB_KERNEL_STAGED) {
        // vw: sites per consumer thread (1 or 2; FP64 1)
        constexpr int S2 = ST == kF64 ? 1 : 2;
        const bool two = ST != kF64 && vw == 2;
        if (p.general == 2) return two ? launch_staged<ST, S2, 2>(p, ctas, s) : launch_staged<ST, 1, 2>(p, ctas, s);
        if (p.general == 1) return two ? launch_staged<ST, S2, 1>(p, ctas, s) : launch_staged<ST, 1, 1>(p, ctas, s);
        return two ? launch_staged<ST, S2, 0>(p, ctas, s) : launch_staged<ST, 1, 0>(p, ctas, s);
    }
    int64_t grid = (ctas > 0 && ctas < p.total_tiles) ? ctas : p.total_tiles;
    if (grid < 1) return cudaSuccess;
    constexpr int V0 = kVW<ST>, V1 = kVW<ST> / 2 > 0 ? kVW<ST> / 2 : 1, V2 = kVW<ST> / 4 > 0 ? kVW<ST> / 4 : 1;
    if (vw == V2)
        k_stream_collide<ST, V2><<<(unsigned)grid, threads, 0, s>>>(p);
    else if (vw == V1)
        k_stream_collide<ST, V1><<<(unsigned)grid, threads, 0, s>>>(p);
    else
        k_stream_collide<ST, V0><<<(unsigned)grid, threads, 0, s>>>(p);
    return cudaGetLastError();
}

template <int ST>
cudaError_t Launch<ST>::bead_couple(const BeadParams& p, int nchains, int max_beads, int lanes, int bpt, cudaStream_t s)
{
    if (nchains <= 0) return cudaSuccess;
    using MT = typename std::conditional<ST == kF64, double, float>::type;
    const size_t dyn = bead_dyn_bytes<MT>(max_beads);
    static int attr_done[kMaxDevices] = {};  // largest dynamic size enabled so far, per device
    cudaError_t e = smem_attr_per_device(k_bead_couple<ST>, (int)dyn, attr_done);
    if (e != cudaSuccess) return e;
    BeadParams q = p;
    q.max_beads = max_beads;
    q.noise_chunk = bead_noise_chunk<MT>(max_beads);
    // MD layout (validated by the caller): lanes per bead and beads per
    // thread; 0 = default, the chain-order layout (two lanes per bead; the
    // autotuner's choice for the 64-bead chain of the 128^3 box: 0.0655 ms per
    // step against 0.0737 ms with eight lanes per bead)
    if (lanes <= 0) {
        lanes = 2;
        bpt = 0;
    }
    if (bpt != 2 && bpt != 0) bpt = 1;
    q.lanes = lanes;
    q.beads_per_thread = bpt;
    // the MD threads, at least 256 for the gather, the noise and the
    // spreading; the chain-order layout: eight threads per bead for those
    int threads = bpt == 0 ? 8 * max_beads : lanes * ((max_beads + bpt - 1) / bpt);
    threads = (threads + 31) / 32 * 32;
    if (threads > kBeadThreadsMax) threads = kBeadThreadsMax;
    if (threads < 256) threads = 256;
    k_bead_couple<ST><<<nchains, threads, dyn, s>>>(q);
    return cudaGetLastError();
}

// A zoomed box's coarse boundary sample onto its face sites (one thread per
// face site and component).
template <class R>
__global__ void k_upsample_faces(const R* coarse, R* fine, int E, int Ec, int z)
{
    const int64_t fe = (int64_t)E * E, total = 18 * fe;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int fc = (int)(i / fe);  // face * 3 + component
        const int64_t r = i - fc * fe;
        const int q = (int)(r / E), p = (int)(r - (int64_t)q * E);
        fine[i] = bilinear_face_site<R>(coarse, Ec, z, fc / 3, fc % 3, p, q);
    }
}

template <int ST>
cudaError_t Launch<ST>::upsample_faces(const void* coarse, void* fine, int E, int Ec, int z, cudaStream_t s)
{
    using R = typename Stor<ST>::R;
    const int64_t total = 18LL * E * E;
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    k_upsample_faces<R><<<blocks, 256, 0, s>>>(reinterpret_cast<const R*>(coarse), reinterpret_cast<R*>(fine), E, Ec, z);
    return cudaGetLastError();
}

template <int ST>
cudaError_t Launch<ST>::forced(const ForcedParams& p, cudaStream_t s)
{
    // a programmatic dependent of the stream-collide before it on the stream:
    // its blocks may start on the SMs that grid has left (they wait on the
    // device for it to complete)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(p.nchains > 0 ? p.nchains * p.splits : 1));
    cfg.blockDim = dim3(kForcedThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_forced<ST>, p);
}

template <int ST>
cudaError_t Launch<ST>::init(void* A, const BoxDev* boxes, int box, int64_t n3, const void* u0, cudaStream_t s)
{
    k_init<ST><<<grid_for(n3, 256), 256, 0, s>>>(reinterpret_cast<typename Stor<ST>::E*>(A), boxes[box],
                                                 reinterpret_cast<const typename Stor<ST>::R*>(u0));
    return cudaGetLastError();
}

template <int ST>
cudaError_t Launch<ST>::fields(const void* A, const BoxDev* boxes, int box, int64_t n3, int what, void* dst,
                               cudaStream_t s)
{
    k_fields<ST><<<grid_for(n3, 256), 256, 0, s>>>(reinterpret_cast<const typename Stor<ST>::E*>(A), boxes[box],
                                                   what, reinterpret_cast<typename Stor<ST>::R*>(dst));
    return cudaGetLastError();
}

template <int ST>
cudaError_t Launch<ST>::read_dev(const void* A, int64_t count, void* dst, cudaStream_t s)
{
    k_read_dev<ST><<<grid_for(count, 256), 256, 0, s>>>(reinterpret_cast<const typename Stor<ST>::E*>(A), count,
                                                        reinterpret_cast<typename Stor<ST>::R*>(dst));
    return cudaGetLastError();
}

template <int ST>
cudaError_t Launch<ST>::conservation(const void* A, const BoxDev* boxes, const ChainDev* chains, int nboxes,
                                     int64_t chunks, const double* vel, double* partial, double* out,
                                     int32_t* status, cudaStream_t s)
{
    dim3 grid((unsigned)chunks, (unsigned)nboxes);
    k_cons_partial<ST><<<grid, kConsThreads, 0, s>>>(A, boxes, chunks, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_cons_final<<<(nboxes + 127) / 128, 128, 0, s>>>(boxes, chains, nboxes, chunks, partial, vel, out, status);
    return cudaGetLastError();
}

}  // namespace lbt
