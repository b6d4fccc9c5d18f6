// Internal structures of the tracer-box library, shared by host and device code.
// Plain structs only; everything here is copied into the caller's device arena.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "lbtracer.h"

namespace lbt {

constexpr int kQ = 19;
constexpr int kRingSlots = 4;       // default ring: samples j-1 .. j+2 live in slots j mod ring_slots
constexpr int kMaxRingSlots = 4096;
// Coarse points per axis of a box with zoom z: point P at site P z, enough
// points to cover site E - 1 (every site when z = 1).
__host__ __device__ inline int coarse_points(int E, int z) { return z > 1 ? (E - 1 + z - 1) / z + 1 : E; }

constexpr int kForcedThreads = 128;  // block of the forced re-collision (one force entry per thread)
constexpr int kMaxBeads = 256;      // beads per chain (one CTA per chain, one thread per bead)

// One box as the kernels see it.
struct BoxDev {
    int64_t f_off;      // element offset of the box's populations in each population buffer
    int64_t n3;         // E^3
    int64_t ring_off;   // element offset of the box's six faces inside one ring slot
    int32_t E;
    int32_t per_mask;   // bit a set: axis a periodic
    int32_t time_interp;
    int32_t K;
    int32_t chain;      // index into the chain table, -1 if none
    int32_t has_accel;
    int32_t zoom;       // coarse grid spacing z in sites (1: samples on every site)
    int32_t Ec;         // coarse points per axis: point P at site P z, covering site E - 1
    int32_t frame;      // 1: frame-acceleration samples add to accel (frame_accel_at)
    int32_t box;        // index of this box in the box table
    int32_t fluct;      // 1: fluctuating collision (FluctDev of the box), 0: BGK
    int32_t fluct_pad;
    uint64_t div_magic; // ceil(2^40 / E): site / E = (site * div_magic) >> 40
    int64_t mlp_row;    // first row of the box in the upsampler output, -1 if the box does not use it
    double tau;
    double rho_b;
    double accel[3];
};

// Body acceleration of box bd at step n: the constant body acceleration plus,
// for a box with frame-acceleration samples, their linear interpolation at
// t_n between samples j = n / K and j + 1 (Sec. 2: the force density
// rho (-dv/dt) of the tracer's co-moving frame).  faccel: [box][slot][4].
__host__ __device__ inline void frame_accel_at(const BoxDev& bd, const double* faccel, int slots, int64_t n,
                                                        double a[3])
{
    for (int c = 0; c < 3; c++) a[c] = bd.accel[c];
    if (!bd.frame) return;
    const int64_t j = n < 0x7fffffff ? (int64_t)((uint32_t)n / (uint32_t)bd.K) : n / bd.K;
    const double th = (double)(n - j * bd.K) / (double)bd.K;
    const double* a0 = faccel + ((int64_t)bd.box * slots + j % slots) * 4;
    const double* a1 = faccel + ((int64_t)bd.box * slots + (j + 1) % slots) * 4;
    for (int c = 0; c < 3; c++) a[c] += (1.0 - th) * a0[c] + th * a1[c];
}

constexpr double kBeadSkin = 0.3;  // Verlet skin of the bead pair lists (lattice units)

// Indices of the per-chain MD constants (ChainDev::md_d / md_f).
enum MdConst {
    kMdDt,        // 1 / n_md
    kMdDtm,       // dt / mass
    kMdNamp,      // noise amplitude sqrt(2 kT zeta / dt), 0 without noise
    kMdR02,       // R0^2
    kMdInvR02,    // 1 / R0^2
    kMdKf,        // FENE k
    kMdZeta,      // friction coefficient
    kMdSig2,      // sigma^2
    kMdRc2,       // WCA cut-off squared, 2^(1/3) sigma^2
    kMdE24,       // 24 eps
    kMdRl2,       // Verlet list radius squared, (2^(1/6) sigma + skin)^2
    kMdHalfSkin2, // (skin / 2)^2
    kMdInvN,      // 1 / nbeads (centre-of-mass averages)
    kMdSkinComp2, // (skin / 2)^2 / 3: per-component displacement bound
    kMdConsts
};

// One chain (bead-spring polymer) as the bead kernel sees it.
struct ChainDev {
    int32_t box;
    int32_t nbeads;     // current chain length (0 until chain_couple)
    int32_t n_md;
    int32_t pin_com;
    int64_t bead_off;   // offset in beads into the position / velocity arrays
    int64_t force_off;  // offset in entries into the force list (8 per bead)
    double k_fene, R0, zeta, mass, kT;
    double eps, sigma;  // WCA repulsion (eps = 0: FENE only)
    double f_ext[3];
    uint64_t seed;
    // MD constants worked out once on the host (FP64 arithmetic is slow on
    // the device), in FP64 and rounded to FP32 for the reduced-precision paths
    double md_d[kMdConsts];
    float md_f[kMdConsts];
};

// Fluctuating collision of one box (lb_set_fluctuation): relaxation factor
// and noise amplitude of the non-conserved modes 4 .. 18 of the D3Q19
// orthogonal basis (see lbt_fluct.cuh).
struct FluctDev {
    uint64_t seed;
    int32_t on;        // 0: the box collides with BGK
    int32_t pad;
    double gamma[15];  // relaxation factor of modes 4 .. 18
    double amp[15];    // sqrt(3 kT b_k (1 - gamma_k^2)); times sqrt(rho) per site
};

// Force density at one lattice site, produced by the bead kernel, consumed by
// the forced re-collision.  site = -1 marks a duplicate of an earlier entry.
struct ForceEntry {
    int32_t site;
    int32_t pad;
    double g[3];
};

// Arena layout (byte offsets), computed by plan().
struct Layout {
    size_t boxes, tile_prefix, chains, pop_a, pop_b, ring, zstage, pos, vel, forces, cons_partial, cons_out,
        status, step, tile_counter, faccel, chain_accel, fluct, mlp_sets, mlp_x, mlp_y, total;
    size_t pop_bytes;        // bytes of one population buffer
    size_t ring_slot_elems;  // real elements per ring slot (6 x 3 x E^2 per box: face sites, zoomed or not)
    int32_t ring_slots;      // slots in the ring of boundary samples
    size_t zstage_bytes;     // staging of the coarse samples of zoomed boxes (6 x 3 x Ec^2 each, back to back)
    int64_t cons_chunks;     // max conservation chunks per box
    int64_t total_beads;
    int64_t mlp_rows;        // face rows of all boxes that use the upsampler
    int32_t mlp_boxes;
    int32_t mlp_K;
};

enum Storage { kF64 = 0, kF32 = 1, kF16 = 2, kBF16 = 3 };

// Parameters of the stream-collide kernel (fused with the boundary layer).
struct SCParams {
    const void* A;
    void* B;
    const void* ring;             // real elements
    int64_t ring_slot_elems;
    int32_t ring_slots;
    const float* mlp_y;           // upsampler output of the current interval, column-major:
    int64_t mlp_ystride;          //   output c of face row r at mlp_y[c * mlp_ystride + r]
    float mlp_yunit;              // velocity of one output unit (u_max / 64)
    const BoxDev* boxes;
    const int64_t* tile_prefix;   // [nboxes + 1] first tile of each box for the current block size
    const double* faccel;         // frame-acceleration samples [box][ring slot][4]
    int32_t general;              // 1: some box is periodic or carries a body force; 2: some box fluctuates
    int32_t nboxes;
    int64_t total_tiles;
    const int64_t* step;          // device step counter n (state holds step n)
    int64_t* tile_counter;        // next tile for the persistent staged kernel (zeroed every step)
    int32_t* status;
    const FluctDev* fluct;        // [nboxes] fluctuating-collision parameters
    int64_t wait_ns;              // limit of the staged kernel's bounded barrier waits
    int64_t withhold_tile;        // test only: the staged producer never arms this tile (-1: none)
    int32_t hint_loads;           // 1: the staged bulk copies take the L2 evict-first policy (chains in the launch)
    int32_t pad_hint;
};

constexpr int64_t kWaitLimitNs = 1000000000;  // bounded device waits give up after one second

// cudaFuncSetAttribute acts on the current device only, so the dynamic
// shared-memory limit of a kernel is raised once per device (and again when a
// launch needs more than before): done[dev] holds the size set on device dev.
constexpr int kMaxDevices = 64;
template <class T>
inline cudaError_t smem_attr_per_device(T* kernel, int bytes, int (&done)[kMaxDevices])
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (done[dev] >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done[dev] = bytes;
    return e;
}

struct BeadParams {
    const void* A;
    const BoxDev* boxes;
    const ChainDev* chains;
    double* pos;
    double* vel;
    ForceEntry* forces;
    const double* faccel;  // frame-acceleration samples [box][ring slot][4]
    double* chain_accel;   // [chain][4]: the body acceleration of the step, for the forced sites
    int32_t ring_slots;
    const int64_t* step;
    int32_t* status;
    int32_t max_beads;    // largest chain of the launch (shared-memory strides)
    int32_t noise_chunk;  // substeps whose noise is drawn at once
    int32_t lanes;        // threads per bead in the MD substeps (1, 2, 4 or 8)
    int32_t beads_per_thread;  // beads an MD thread holds (1 or 2; 0: chain order, two lanes per bead)
    double* hist;              // chain trajectory ring (null: off): [slot][3 x total beads]
    int64_t hist_stride;       // doubles per slot
    int32_t hist_slots;
    int32_t hist_pad;
};

struct ForcedParams {
    const void* A;
    void* B;
    const BoxDev* boxes;
    const ChainDev* chains;
    const ForceEntry* forces;
    const double* chain_accel;    // [chain][4], written by the bead kernel of the step
    const int32_t* status;
    int64_t* step;                // incremented once per step by block 0
    int64_t* tile_counter;        // reset to zero once per step by block 0
    int32_t nchains;
    int32_t splits;               // blocks per chain (set by the launcher)
};

// Mean |curl u| over the cube [lo, hi]^3 of a velocity field u [3][E^3]
// (double when u_f64, else float); scratch holds 513 doubles, out one double
// (both device memory).
cudaError_t launch_vorticity(const void* u, int u_f64, int E, int lo, int hi, double* scratch, double* out,
                             cudaStream_t s);

// Host-side launchers, one instantiation per storage type.
template <int ST>
struct Launch {
    static cudaError_t stream_collide(const SCParams& p, int kernel, int threads, int ctas, int vw, cudaStream_t s);
    static cudaError_t bead_couple(const BeadParams& p, int nchains, int max_beads, int lanes, int bpt, cudaStream_t s);
    // coarse face sample [6][3][Ec][Ec] -> face sites [6][3][E][E] (bilinear, point P at site P z)
    static cudaError_t upsample_faces(const void* coarse, void* fine, int E, int Ec, int z, cudaStream_t s);
    static cudaError_t forced(const ForcedParams& p, cudaStream_t s);
    static cudaError_t init(void* A, const BoxDev* boxes, int box, int64_t n3, const void* u0, cudaStream_t s);
    static cudaError_t fields(const void* A, const BoxDev* boxes, int box, int64_t n3, int what, void* dst,
                              cudaStream_t s);
    static cudaError_t read_dev(const void* A, int64_t count, void* dst, cudaStream_t s);
    static cudaError_t conservation(const void* A, const BoxDev* boxes, const ChainDev* chains, int nboxes,
                                    int64_t chunks, const double* vel, double* partial, double* out,
                                    int32_t* status, cudaStream_t s);
};

// Generator launchers; workspace holds the per-axis phase table (3 M E double2).
// Points: every zoom-th site, (E - 1)/zoom + 1 per axis.
cudaError_t launch_synth_faces(const double* kvec, const double* amp, const double* omega, const double* phi,
                               int M, int E, int zoom, int K, int64_t j0, int64_t nsamp, int out_f64, void* out,
                               void* workspace, cudaStream_t s);
cudaError_t launch_synth_volume(const double* kvec, const double* amp, const double* omega, const double* phi,
                                int M, int E, int zoom, double t, int out_f64, void* out, void* workspace,
                                cudaStream_t s);

}  // namespace lbt

// Message returned by lb_last_error(NULL) for calls that have no context.
void lbt_set_last_error(const char* msg);

// Sites per tile of the staged stream-collide kernel for a storage format.
int lbt_staged_tile_sites(int spt);               // sites per tile of the staged kernel
bool lbt_staged_spt_ok(int storage, int spt);      // staged sites per consumer thread supported
int lbt_staged_default_spt(int storage);
