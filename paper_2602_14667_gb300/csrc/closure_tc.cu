// closure_tc.cu -- the closure step (learned correction of a1^(2); the
// closure is not part of the paper) with its MLP on the 5th-generation
// tensor cores (tcgen05).
//
// The walk is that of step_closure_rows: a warp takes one tile of 30 output
// columns (lanes 0 and 31 hold the neighbouring columns) and a stack of rows,
// pulls every row of the walk into a per-warp stage of three row slots by
// cp.async one row ahead of its use, keeps u and b of three rows in
// registers and forms the 24 features of the row before the newest one.
// Here the four warps of a warpgroup walk four tiles side by side, so that
// their 4 x 32 feature rows are one M = 128 block: they write them as the
// K-major layer-1 operand in shared memory, one thread issues tcgen05.mma
// for each layer (FP32 accumulators in 64 tensor-memory columns, 128 lanes:
// one row per lane), and every warp reads back its own 32 lanes, adds the
// bias, applies ReLU and writes the next layer's operand.  The two
// warpgroups of a block run independently; the only block-wide barriers are
// the one after the weights are staged and the one at exit.  Every wait on
// the tensor cores is bounded: a wait that gives up sets *err (reported as
// MHD_ECUDA) and ends the warpgroup's walk, and the tensor memory is freed on
// every path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstddef>
#include <cstdint>

#include "closure_device.cuh"
#include "closure_internal.h"
#include "tc_ops.cuh"

namespace mhd {

namespace {

constexpr int kTW = 8;                  // warps per block: two warpgroups, each one M = 128 block
constexpr int kN3 = 16;                 // layer-3 N (3 outputs, padded)
constexpr int kTmemCols = 128;          // two M = 128 x N = 64 accumulators
constexpr int kMbarWaitLimit = 1 << 17; // x <= ~1 us: a wait gives up after ~0.1 s

struct RowsTcShared {
    // operands in the K-major core-matrix layout of tc_ops.cuh
    alignas(128) unsigned char W1[kHid * kInPad * 2];  // 64 x 32
    alignas(128) unsigned char W2[kHid * kHid * 2];    // 64 x 64
    alignas(128) unsigned char W3[kN3 * kHid * 2];     // 16 x 64 (rows >= kOutPad zero)
    // per M block: the 128 x 32 features of layer 1, then the 128 x 64
    // activations of layers 2 and 3
    alignas(128) unsigned char act[2][128 * kHid * 2];
    alignas(16) float b1[kHid];
    alignas(16) float b2[kHid];
    float b3[kOutPad];
    alignas(16) float mean[kIn];
    alignas(16) float scale[kIn];
    float out_scale[kOut];
    float stage[kTW][3][kPlanes][32];  // per warp: three pulled rows, plane-major, a column per lane
    alignas(8) uint64_t mbar[2];       // one per M block
    uint32_t tmem;
};
static_assert(offsetof(RowsTcShared, W1) % 128 == 0 && offsetof(RowsTcShared, W2) % 128 == 0 &&
                  offsetof(RowsTcShared, W3) % 128 == 0 && offsetof(RowsTcShared, act) % 128 == 0,
              "tensor-core operands must be 16-byte aligned");
static_assert(offsetof(RowsTcShared, mbar) % 8 == 0, "mbarrier alignment");
static_assert(2 * (sizeof(RowsTcShared) + 1024) <= 228 * 1024, "two blocks per SM");

// Issue one MLP layer of M block h (one thread) and make the block's
// mbarrier arrive when it completes.  A: act[h] with K columns; B: N x K.
template <int K, int N>
__device__ __forceinline__ void issue_layer(RowsTcShared& sh, int h, const unsigned char* B, uint32_t tmem) {
    constexpr uint32_t sbo = (K / 8) * 128, idesc = tc::idesc_bf16(128, N);
    const uint32_t a0 = tc::smem_u32(sh.act[h]), b0 = tc::smem_u32(B);
#pragma unroll
    for (int s = 0; s < K / 16; ++s)
        tc::mma_bf16(tmem + 64 * h, tc::smem_desc(a0 + 256 * s, 128, sbo), tc::smem_desc(b0 + 256 * s, 128, sbo),
                     idesc, s);
    tc::commit(&sh.mbar[h]);
}

// barrier of the 128 threads (4 warps) of M block h; returns whether any of
// them passed `pred`
template <int ID>
__device__ __forceinline__ bool bar_or_128(bool pred) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, 128, p;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "n"(ID)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ bool group_bar_or(int h, bool pred) {
    return h == 0 ? bar_or_128<1>(pred) : bar_or_128<2>(pred);
}

// ReLU(acc + bias) of this thread's row (64 columns of its tensor-memory
// lane), rounded to BF16, into row `row` of the K = 64 operand of block h.
__device__ __forceinline__ void relu_to_act(RowsTcShared& sh, int h, const float* bias, uint32_t taddr, int row) {
#pragma unroll
    for (int c = 0; c < kHid; c += 32) {
        float v[32];
        tc::ld32(taddr + c, v);
#pragma unroll
        for (int q = 0; q < 32; q += 8) {
            const float4 b0 = *reinterpret_cast<const float4*>(bias + c + q);
            const float4 b1 = *reinterpret_cast<const float4*>(bias + c + q + 4);
            const uint4 w = make_uint4(relu_pack2(v[q] + b0.x, v[q + 1] + b0.y), relu_pack2(v[q + 2] + b0.z, v[q + 3] + b0.w),
                                       relu_pack2(v[q + 4] + b1.x, v[q + 5] + b1.y),
                                       relu_pack2(v[q + 6] + b1.z, v[q + 7] + b1.w));
            *reinterpret_cast<uint4*>(sh.act[h] + tc::canon_off(row, c + q, kHid)) = w;
        }
    }
}

template <typename Off>
__global__ void __launch_bounds__(kTW * 32, 2) step_closure_rows_tc(const StepArgs<float> a, const ClosureParamsDev cp,
                                                                    int strips, int rows, int ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RowsTcShared& sh = *reinterpret_cast<RowsTcShared*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int h = warp >> 2, hrow = tid & 127;  // this warp's M block and this thread's row in it
    const float* src = static_cast<const float*>(a.src);
    float* dst = static_cast<float*>(a.dst);
    // the network, in 16-byte pieces, into the operand layout
    constexpr int kC1 = kInPad / 8, kC2 = kHid / 8;  // 16-byte pieces per weight row
    for (int i = tid; i < kHid * kC1; i += kTW * 32)
        cp_async16(sh.W1 + tc::canon_off(i / kC1, 8 * (i % kC1), kInPad), cp.Wt1 + (i / kC1) * kInPad + (i % kC1) * 8);
    for (int i = tid; i < kHid * kC2; i += kTW * 32)
        cp_async16(sh.W2 + tc::canon_off(i / kC2, 8 * (i % kC2), kHid), cp.Wt2 + (i / kC2) * kHid + (i % kC2) * 8);
    for (int i = tid; i < kOutPad * kC2; i += kTW * 32)
        cp_async16(sh.W3 + tc::canon_off(i / kC2, 8 * (i % kC2), kHid), cp.Wt3 + (i / kC2) * kHid + (i % kC2) * 8);
    cp_async_commit();
    for (int i = tid; i < (kN3 - kOutPad) * kC2; i += kTW * 32)
        *reinterpret_cast<uint4*>(sh.W3 + tc::canon_off(kOutPad + i / kC2, 8 * (i % kC2), kHid)) = make_uint4(0, 0, 0, 0);
    if (tid < kHid) { sh.b1[tid] = cp.b1[tid]; sh.b2[tid] = cp.b2[tid]; }
    if (tid < kOutPad) sh.b3[tid] = cp.b3[tid];
    if (tid < kIn) { sh.mean[tid] = cp.mean[tid]; sh.scale[tid] = cp.scale[tid]; }
    if (tid < kOut) sh.out_scale[tid] = cp.out_scale[tid];

    // tile t: strip t % strips of 30 output columns (lane l holds column
    // 30 * strip - 1 + l, wrapped), rows [y0, y1) of segment t / strips; row
    // i of its walk is y0 - 1 + i (even segments) or y1 - i (odd ones)
    struct Tile {
        int xl, xw, y0, y1;
        bool up;
    };
    auto tile_of = [&](int t) {
        Tile T;
        const int strip = t % strips, seg = t / strips;
        T.xl = strip * 30 - 1 + lane;
        T.xw = T.xl % a.nx;
        if (T.xw < 0) T.xw += a.nx;
        T.y0 = seg * rows;
        T.y1 = min(a.ny, T.y0 + rows);
        T.up = seg & 1;
        return T;
    };
    // the pull of row i of tile T into stage slot sl: each lane copies its
    // own node's 19 cells into its own column of the slot
    auto issue_row = [&](const Tile& T, int i, int sl) {
        const int m = T.up ? T.y1 - i : T.y0 - 1 + i;
        const int my = m < 0 ? m + a.ny : (m >= a.ny ? m - a.ny : m);
        const int ym = my == 0 ? a.ny - 1 : my - 1, yp = my + 1 == a.ny ? 0 : my + 1;
        const int xm = T.xw == 0 ? a.nx - 1 : T.xw - 1, xp = T.xw + 1 == a.nx ? 0 : T.xw + 1;
        const Off pt = (Off)a.pitch, pl = (Off)a.plane;
        const Off r_m = (Off)ym * pt, r_0 = (Off)my * pt, r_p = (Off)yp * pt;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const int cx = pcx(p), cy = pcy(p);
            const Off o = (Off)p * pl + (cy > 0 ? r_m : (cy < 0 ? r_p : r_0)) + (cx > 0 ? xm : (cx < 0 ? xp : T.xw));
            cp_async4(&sh.stage[warp][sl][p][lane], src + o);
        }
    };
    // The four warps of warpgroup g = 2 blockIdx + h walk tiles 4 g + (warp
    // & 3), then those ngroups groups further on; every warp of the group
    // runs the same rows + 2 row iterations per group tile (a warp whose
    // tile is shorter, or absent, idles through the MMAs of the others).
    const int ngroups = 2 * gridDim.x;
    int tg = 2 * blockIdx.x + h;
    auto wtile = [&](int g) { return 4 * g + (warp & 3); };
    // the first row of the warp's first tile is in flight while the weights land
    if (wtile(tg) < ntiles) issue_row(tile_of(wtile(tg)), 0, 0);
    cp_async_commit();
    if (warp == 0) tc::tmem_alloc<kTmemCols>(&sh.tmem);
    if (tid == 0) { tc::mbar_init(&sh.mbar[0], 1); tc::mbar_init(&sh.mbar[1], 1); }
    cp_async_wait<1>();  // this thread's weight pieces (the older group)
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sh.tmem;
    const uint32_t tlane = tmem + 64 * h + ((uint32_t)(32 * (warp & 3)) << 16);
    unsigned char* A = sh.act[h];
    const bool out_lane = lane >= 1 && lane <= 30;
    const float rho0 = a.np.rho0;
    uint32_t phase = 0;
    bool failed = false;
    int sl = 0;  // stage slot of the row about to be used
    for (; 4 * tg < ntiles && !failed; tg += ngroups) {
        const int t = wtile(tg), tn = wtile(tg + ngroups);
        const bool have = t < ntiles;
        const Tile T = tile_of(have ? t : 0);
        const int nrow = have ? T.y1 - T.y0 + 2 : 0;
        const float sgn = T.up ? -1.f : 1.f;
        float wnd[3][4] = {};  // u_x, u_y, b_x, b_y of the last three rows (slot 2 newest)
        for (int i = 0; i < rows + 2; ++i) {
            const bool real = i < nrow;  // this warp's walk has a row i
            const int sl_next = sl == 2 ? 0 : sl + 1, sl_prev = sl == 0 ? 2 : sl - 1;
            if (real) {
                if (i + 1 < nrow)
                    issue_row(T, i + 1, sl_next);
                else if (4 * (tg + ngroups) < ntiles && tn < ntiles)
                    issue_row(tile_of(tn), 0, sl_next);
            }
            cp_async_commit();
            cp_async_wait<1>();
            const float(*cur)[32] = sh.stage[warp][sl_prev];
            if (real) {
                const float(*nxt)[32] = sh.stage[warp][sl];
                sl = sl_next;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    wnd[0][q] = wnd[1][q];
                    wnd[1][q] = wnd[2][q];
                }
                float f[9], g[10];
#pragma unroll
                for (int k = 0; k < 9; ++k) f[k] = nxt[k][lane];
#pragma unroll
                for (int k = 0; k < 10; ++k) g[k] = nxt[9 + k][lane];
                const Moments<float> mm = moments(f, g, rho0);
                wnd[2][0] = mm.ux;
                wnd[2][1] = mm.uy;
                wnd[2][2] = mm.bx;
                wnd[2][3] = mm.by;
            }
            if (i < 2) continue;  // uniform over the warpgroup
            // the features of this warp's row i - 1 (zero rows when it has none)
            {
                uint32_t pk[kInPad / 2];
#pragma unroll
                for (int c = 0; c < kInPad / 2; ++c) pk[c] = 0u;
                if (real) {
                    float fe[kIn];
                    float f[9], g[10];
#pragma unroll
                    for (int k = 0; k < 9; ++k) f[k] = cur[k][lane];
#pragma unroll
                    for (int k = 0; k < 10; ++k) g[k] = cur[9 + k][lane];
                    point_features(f, g, rho0, fe);
                    stencil_rows(wnd, sgn, fe + 8);
#pragma unroll
                    for (int c4 = 0; c4 < kIn / 4; ++c4) {
                        const float4 mu = *reinterpret_cast<const float4*>(sh.mean + 4 * c4);
                        const float4 sc = *reinterpret_cast<const float4*>(sh.scale + 4 * c4);
                        pk[2 * c4] = pack2((fe[4 * c4] - mu.x) * sc.x, (fe[4 * c4 + 1] - mu.y) * sc.y);
                        pk[2 * c4 + 1] = pack2((fe[4 * c4 + 2] - mu.z) * sc.z, (fe[4 * c4 + 3] - mu.w) * sc.w);
                    }
                }
#pragma unroll
                for (int c = 0; c < kInPad / 8; ++c)
                    *reinterpret_cast<uint4*>(A + tc::canon_off(hrow, 8 * c, kInPad)) =
                        make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
            }
            // three layers of this M block: operand writes -> async proxy,
            // the block's first thread issues, its 128 threads wait
            float out[kN3];
#pragma unroll 1
            for (int layer = 0; layer < 3; ++layer) {
                tc::fence_smem_to_async();
                tc::fence_before_sync();
                group_bar_or(h, false);
                tc::fence_after_sync();
                if (hrow == 0) {
                    if (layer == 0) issue_layer<kInPad, kHid>(sh, h, sh.W1, tmem);
                    else if (layer == 1) issue_layer<kHid, kHid>(sh, h, sh.W2, tmem);
                    else issue_layer<kHid, kN3>(sh, h, sh.W3, tmem);
                }
                const bool ok = tc::mbar_wait(&sh.mbar[h], phase, kMbarWaitLimit);
                phase ^= 1;
                tc::fence_after_sync();
                if (group_bar_or(h, !ok)) {
                    failed = true;
                    break;
                }
                if (layer == 0) relu_to_act(sh, h, sh.b1, tlane, hrow);
                else if (layer == 1) relu_to_act(sh, h, sh.b2, tlane, hrow);
                else tc::ld16(tlane, out);
            }
            if (failed) break;
            if (real && out_lane && T.xl < a.nx) {
                const int o = T.up ? T.y1 - i + 1 : T.y0 - 2 + i;  // the row of cur: y0 <= o < y1
                float f[9], g[10];
#pragma unroll
                for (int k = 0; k < 9; ++k) f[k] = cur[k][lane];
#pragma unroll
                for (int k = 0; k < 10; ++k) g[k] = cur[9 + k][lane];
                const float d3[3] = {(out[0] + sh.b3[0]) * sh.out_scale[0], (out[1] + sh.b3[1]) * sh.out_scale[1],
                                     (out[2] + sh.b3[2]) * sh.out_scale[2]};
                if (cp.da_out) {
                    const Off nn = (Off)a.nx * (Off)a.ny, node = (Off)o * (Off)a.nx + T.xl;
#pragma unroll
                    for (int k = 0; k < 3; ++k) cp.da_out[(Off)k * nn + node] = d3[k];
                }
                collide_impl<true, float>(f, g, a.np, d3);
                const Off off = (Off)o * (Off)a.pitch + T.xl, pl = (Off)a.plane;
#pragma unroll
                for (int k = 0; k < 9; ++k) dst[(Off)k * pl + off] = f[k];
#pragma unroll
                for (int k = 0; k < 10; ++k) dst[(Off)(9 + k) * pl + off] = g[k];
            }
        }
    }
    // every thread arrives here; a warpgroup may have given up
    if (__syncthreads_or(failed)) {
        if (tid == 0) atomicExch(cp.err, 1);
        // the MMAs of a warpgroup that gave up may still be running: wait
        // for them (bounded) before the tensor memory is given back
        if (failed) tc::mbar_wait(&sh.mbar[h], phase ^ 1, kMbarWaitLimit);
    }
    cp_async_wait<0>();  // nothing left in flight when the block exits
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free<kTmemCols>(tmem);
}

}  // namespace

cudaError_t launch_step_closure_tc(const StepLaunch& s, const ClosureParamsDev& cp, cudaStream_t st) {
    if (s.prec != 1 || s.wall_x || s.wall_y) return cudaErrorInvalidValue;
    // the weight blocks are staged in 16-byte pieces
    for (const void* w : {(const void*)cp.Wt1, (const void*)cp.Wt2, (const void*)cp.Wt3})
        if (reinterpret_cast<uintptr_t>(w) % 16) return cudaErrorInvalidValue;
    if (!cp.err) return cudaErrorInvalidValue;
    StepArgs<float> a;
    a.src = s.src;
    a.dst = s.dst;
    a.nx = s.L.nx;
    a.ny = s.L.ny;
    a.pitch = s.L.pitch;
    a.plane = s.L.plane;
    a.np.omega = (float)s.omega;
    a.np.omega_m = (float)s.omega_m;
    a.np.rho0 = (float)s.rho0;
    a.np.variant = s.variant;
    a.np.collision = s.collision;
    a.np.mag_collision = s.mag_collision;
    a.wall_x = 0;
    a.wall_y = 0;
    const size_t smem = sizeof(RowsTcShared);
    // int element offsets while the 19 planes hold fewer than 2^31 elements
    const bool small = (long long)kPlanes * s.L.plane < (1LL << 31);
    auto kernel = small ? step_closure_rows_tc<int> : step_closure_rows_tc<long long>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // all of the unified L1 / shared storage as shared memory, so that two
    // blocks fit on an SM
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int sms = 0, dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // Two blocks per SM (registers by the launch bounds, shared memory by
    // the static_assert; 2 x 128 of the 512 tensor-memory columns; the
    // occupancy calculator answers one for a kernel that allocates tensor
    // memory).  Tiles as for step_closure_rows: strips of 30 columns, row
    // segments so that the tiles are about as many as the resident warps,
    // and a whole number of warpgroups' worth of tiles in flight.
    const long long strips = (s.L.nx + 29) / 30;
    const long long maxb = 2LL * sms;
    const long long segs_want = std::max(1LL, maxb * kTW / strips);
    const long long rows = ((long long)s.L.ny + segs_want - 1) / segs_want;
    const long long segs = ((long long)s.L.ny + rows - 1) / rows;
    const long long ntiles = strips * segs;
    if (ntiles > (1LL << 30) || rows > INT_MAX / 2) return cudaErrorInvalidValue;
    const int blocks = (int)std::max(1LL, std::min(maxb, (ntiles + kTW - 1) / kTW));
    kernel<<<blocks, kTW * 32, smem, st>>>(a, cp, (int)strips, (int)rows, (int)ntiles);
    return cudaGetLastError();
}

}  // namespace mhd
