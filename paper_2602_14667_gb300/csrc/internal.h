// internal.h -- host-side declarations shared by the library's translation
// units (kernel launchers and layout).  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <string>

namespace mhd {

constexpr int kStatePlanes = 19;  // 9 f_i + 5 x 2 g_{j,a} per buffer

// Geometry of one population buffer: 19 planes of ny rows x pitch elements.
struct Layout {
    int nx, ny;
    long long pitch;  // elements per row (multiple of 128 bytes)
    long long plane;  // elements per plane (ny * pitch rounded to 256 bytes)
    int esize;        // bytes per stored element (8, 4, 2)
};

// Everything a step launch needs.  Doubles are converted to the compute
// type inside the launcher.
struct StepLaunch {
    Layout L;
    int prec;  // 0 fp64, 1 fp32, 2 fp16s
    const void* src;
    void* dst;
    double omega, omega_m, rho0;
    int variant, collision, mag_collision, wall_x, wall_y;
    int V;      // nodes per thread along x
    int BY;     // warps (rows) per block
    int W = 0;  // resident warps per SM of the persistent grid (0: step_rule_warps)
};

// fused stream + collide (one time step)
cudaError_t launch_step(const StepLaunch& s, cudaStream_t st);
// is (V, BY) a legal launch shape for this lattice?
bool step_shape_ok(const Layout& L, int prec, int wall_x, int V, int BY);
// The built-in staging depth of the row kernels: resident warps per SM that
// keep about 4 KB of every plane in flight (warps x 32 lanes x V elements);
// FP64, bound by its arithmetic, keeps every resident warp (64).
int step_rule_warps(int prec, int V);

// f = f_eq(rho, u, b), g = g_eq(u, b) from FP64 (or FP32) fields in device
// memory or in mapped pinned host memory (rho may be null); with flags, the
// input checks of mhd_set_fields OR-ed into *flags (the state is written
// either way)
cudaError_t launch_init(const Layout& L, int prec, void* buf, const double* rho, const double* ux,
                        const double* uy, const double* bx, const double* by, double rho0,
                        int variant, cudaStream_t st, int* flags = nullptr);
cudaError_t launch_init(const Layout& L, int prec, void* buf, const float* rho, const float* ux,
                        const float* uy, const float* bx, const float* by, double rho0, int variant,
                        cudaStream_t st, int* flags = nullptr);
// rho, u, b (FP64, or FP64 rounded to FP32; nx*ny each, any may be null)
// of the stored state, into device memory or mapped pinned host memory
cudaError_t launch_fields(const Layout& L, int prec, const void* buf, double rho0, double* rho,
                          double* ux, double* uy, double* bx, double* by, cudaStream_t st);
cudaError_t launch_fields(const Layout& L, int prec, const void* buf, double rho0, float* rho, float* ux,
                          float* uy, float* bx, float* by, cudaStream_t st);
// planes of one slab exchange (up to all 19)
struct HaloPlanes {
    int p[kStatePlanes];
    int n;
};
// one launch for the row copies of a slab exchange on one device (see
// halo_rows_kernel); cudaErrorInvalidValue unless every size, offset and
// base address is a multiple of 16 bytes
cudaError_t launch_halo_rows(const void* src, void* dst, long long src_plane, long long dst_plane, long long src_off,
                             long long dst_off, long long bytes, const HaloPlanes& hp, cudaStream_t st);
// one copy of a slab group's exchange: the 5 crossing planes of one padded
// row, src and dst already at the row (plane 0), plane strides in bytes
struct HaloJob {
    const char* src;
    char* dst;
    long long src_plane, dst_plane;
    int planes[5];
};
// every job of a device job table in one launch (row_bytes a multiple of
// 16; cudaErrorInvalidValue otherwise)
cudaError_t launch_halo_jobs(const HaloJob* jobs, int njobs, long long row_bytes, cudaStream_t st);
// stored state whose pull-gather reproduces the packed FP32 pre-collision
// state F (periodic axes)
cudaError_t launch_unstream(const Layout& L, int prec, void* buf, const float* F, cudaStream_t st);
// one plane <-> unshifted FP64 array of nx*ny (population p = 0..18)
cudaError_t launch_plane_out(const Layout& L, int prec, const void* buf, int p, double rho0,
                             double* out, cudaStream_t st);
cudaError_t launch_plane_in(const Layout& L, int prec, void* buf, int p, double rho0,
                            const double* in, cudaStream_t st);

// Diagnostics.  mode 0: gather the pre-collision state from `prev` (the
// buffer the last step read); mode 1: use `cur` in place, with the
// magnetic non-equilibrium scaled by neq_scale.  A persistent grid of at
// most `capacity` blocks walks strip tiles of the lattice; each block
// writes kDiagSlots doubles into `partials` (room for `capacity` blocks),
// then they are reduced in a fixed order into `totals` (kDiagSlots
// doubles).  diag_blocks(L) is a capacity that never limits the grid.
constexpr int kDiagSlots = 13;
struct DiagLaunch {
    Layout L;
    int prec;
    const void* prev;
    const void* cur;
    int mode;
    double omega_m, rho0, neq_scale;
    int wall_x, wall_y;
    int halo_y = 0;  // slab: rows -1 and ny are ghost rows of `cur` (mode 1 only)
};
int diag_blocks(const Layout& L);
cudaError_t launch_diag(const DiagLaunch& d, double* partials, int capacity, double* totals, cudaStream_t st);
// The fixed-order reduction of `nblocks` per-block partials into `totals`
// (slot 0 plus mass_base: the mass).
cudaError_t launch_diag_final(const double* partials, int nblocks, double mass_base, double* totals,
                              cudaStream_t st);

// The diagnostics of a whole ensemble (FP32 storage, periodic lattices) in
// one launch over a list of (lattice, tile) pairs, then one block per
// lattice adding its tiles' partials in order.  DiagEnsemble holds the
// device tables, built once for the ensemble's layouts.
struct DiagEnsemble {
    int count = 0, ntiles = 0;
    void* d_args = nullptr;   // per-lattice kernel arguments, refreshed by every launch
    void* h_args = nullptr;   // their pinned host staging
    void* d_tiles = nullptr;  // (lattice, tile) pairs
    int* d_first = nullptr;   // first tile of each lattice (count + 1)
    double* d_mass = nullptr;  // rho0 * nodes of each lattice
    double* d_partials = nullptr;  // kDiagSlots per tile
};
// What one lattice of the ensemble reduces now: the buffer the last step
// read (mode 0, gathered) or the stored state (mode 1, with neq_scale).
struct DiagLatticeState {
    const void* prev;
    const void* cur;
    int mode;
    double omega_m, rho0, neq_scale;
};
cudaError_t diag_ensemble_create(DiagEnsemble& e, const Layout* layouts, const double* rho0, int count);
void diag_ensemble_destroy(DiagEnsemble& e);
// cudaErrorNotSupported when a lattice does not allow the two-node vector
// loads (odd nx, or rows not 8-byte aligned): take launch_diag per lattice.
// totals: kDiagSlots doubles per lattice.
cudaError_t diag_ensemble_launch(DiagEnsemble& e, const Layout* layouts, const DiagLatticeState* states,
                                 double* totals, cudaStream_t st);
// Lattice l's totals (kDiagSlots doubles at totals + kDiagSlots l) from its
// tiles' partials [first[l], first[l + 1]) added in order; slot 0 plus
// mass_base[l] is the mass.
cudaError_t launch_diag_batch_final(const double* tile_partials, const int* first, const double* mass_base,
                                    int count, double* totals, cudaStream_t st);

// One step (as launch_step, two buffers, periodic x; s.V nodes per lane)
// that also reduces the point totals of the pre-collision state it gathers
// into `totals` (kDiagSlots doubles, the diagnostics' slots; the slots of
// the gradient quantities, 8, 9, 10 and 12, are zero) through at most
// `capacity` per-block partials.  The populations it writes are those of
// launch_step.  cudaErrorInvalidValue for x walls.
cudaError_t launch_step_totals(const StepLaunch& s, double* partials, int capacity, double* totals,
                               cudaStream_t st);

Layout make_layout(int nx, int ny, int prec);

// SM count of the current device (queried once per device; 152 on GB300 if
// the query fails).  Grid-stride launchers size their grids with it.
int device_sms();

// message returned by mhd_last_error() in the calling thread
void set_last_error(const std::string& msg);

}  // namespace mhd
