// closure_tc.cu -- the closure step with its MLP on the 5th-generation
// tensor cores (tcgen05): per 32 x 8-node tile the 256 feature rows form two
// M = 128 blocks; one thread per block issues tcgen05.mma on shared-memory
// operands, the accumulators sit in tensor memory (128 of its columns per
// thread block), and every warp reads back the rows of its own 32 nodes,
// applies bias and ReLU and writes the next layer's operand.  The gather,
// features and collision are those of the warp-MMA closure step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "closure_device.cuh"
#include "closure_internal.h"
#include "tc_ops.cuh"

namespace mhd {

// The MLP runs on the 5th-generation tensor cores: per 32 x 8-node tile the
// 256 feature rows are two M = 128 blocks; one thread issues tcgen05.mma on
// shared-memory operands, the accumulators sit in tensor memory (128 of its
// columns per block), and every warp reads back the rows of its own 32 nodes.
constexpr int kN3 = 16;                            // layer-3 N (3 outputs, padded)
constexpr int kTmemCols = 128;                     // two M = 128 x N = 64 accumulators
constexpr int kMbarWaitLimit = 1 << 17;            // x <= ~1 us: a wait gives up after ~0.1 s

struct ClosureSharedTC {
    // operands in the K-major core-matrix layout of tc_ops.cuh
    alignas(128) unsigned char W1[kHid * kInPad * 2];  // 64 x 32
    alignas(128) unsigned char W2[kHid * kHid * 2];    // 64 x 64
    alignas(128) unsigned char W3[kN3 * kHid * 2];     // 16 x 64 (rows >= kOutPad zero)
    // per M block of 128 nodes (16 KB each): the 128 x 32 features of layer
    // 1, then the 128 x 64 activations of layers 2 and 3
    alignas(128) unsigned char act[2][128 * kHid * 2];
    float b1[kHid], b2[kHid], b3[kOutPad];
    float mean[kIn], scale[kIn], out_scale[kOut];
    float mom[4][kCHY][kCHX];
    // pre-collision populations of the tile and of its halo ring, double
    // buffered: cp.async fills one while the other tile is processed
    float pop[2][kPlanes][kTile];
    float hpop[2][kPlanes][kHalo];
    alignas(8) uint64_t mbar[2];  // one per M block
    uint32_t tmem;
};
static_assert(offsetof(ClosureSharedTC, W1) % 128 == 0 && offsetof(ClosureSharedTC, W2) % 128 == 0 &&
                  offsetof(ClosureSharedTC, W3) % 128 == 0 && offsetof(ClosureSharedTC, act) % 128 == 0,
              "tensor-core operands must be 16-byte aligned");
static_assert(offsetof(ClosureSharedTC, mbar) % 8 == 0, "mbarrier alignment");
static_assert(sizeof(((ClosureSharedTC*)nullptr)->act[0]) == 128 * kHid * 2, "one M block of activations");
static_assert(2 * (sizeof(ClosureSharedTC) + 1024) <= 228 * 1024, "two blocks per SM");

// Issue one MLP layer of M block h (one thread) and make the block's
// mbarrier arrive when it completes.  A: act[h] with K columns; B: N x K.
template <int K, int N>
__device__ __forceinline__ void issue_layer(ClosureSharedTC& sh, int h, const unsigned char* B, uint32_t tmem) {
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
__device__ __forceinline__ bool half_bar_or(int h, bool pred) {
    return h == 0 ? bar_or_128<1>(pred) : bar_or_128<2>(pred);
}

// ReLU(acc + bias) of this thread's node (64 columns of its tensor-memory
// lane) as bf16 into row `row` of the K = 64 activation operand of block h.
__device__ __forceinline__ void relu_to_act(ClosureSharedTC& sh, int h, const float* bias, uint32_t taddr, int row) {
#pragma unroll
    for (int c = 0; c < kHid; c += 32) {
        float v[32];
        tc::ld32(taddr + c, v);
#pragma unroll
        for (int q = 0; q < 32; q += 8) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                w[j] = pack2(fmaxf(v[q + 2 * j] + bias[c + q + 2 * j], 0.f),
                             fmaxf(v[q + 2 * j + 1] + bias[c + q + 2 * j + 1], 0.f));
            *reinterpret_cast<uint4*>(sh.act[h] + tc::canon_off(row, c + q, kHid)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Persistent 32 x 8-node tiles.  The populations of the next tile are
// gathered by cp.async into the other buffer while this tile's features,
// MLP (tensor cores) and collision run.  The two M blocks of a tile (warps
// 0-3 and 4-7) run their three layers independently, so one block's
// epilogue overlaps the other's MMAs.  A tensor-core wait that gives up
// sets *err and ends the kernel (the tensor memory is still freed).
__global__ void __launch_bounds__(256, 2) step_closure_tc(const StepArgs<float> a, const ClosureParamsDev cp,
                                                       int ntx, int ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ClosureSharedTC& sh = *reinterpret_cast<ClosureSharedTC*>(smem_raw);
    const int tid = threadIdx.y * kCTX + threadIdx.x, lane = threadIdx.x, ly = threadIdx.y;
    const float* src = static_cast<const float*>(a.src);
    float* dst = static_cast<float*>(a.dst);
    // the network, in 16-byte pieces, into the operand layout
    constexpr int kC1 = kInPad / 8, kC2 = kHid / 8;  // 16-byte pieces per weight row
    for (int i = tid; i < kHid * kC1; i += kTile)
        cp_async16(sh.W1 + tc::canon_off(i / kC1, 8 * (i % kC1), kInPad), cp.Wt1 + (i / kC1) * kInPad + (i % kC1) * 8);
    for (int i = tid; i < kHid * kC2; i += kTile)
        cp_async16(sh.W2 + tc::canon_off(i / kC2, 8 * (i % kC2), kHid), cp.Wt2 + (i / kC2) * kHid + (i % kC2) * 8);
    for (int i = tid; i < kOutPad * kC2; i += kTile)
        cp_async16(sh.W3 + tc::canon_off(i / kC2, 8 * (i % kC2), kHid), cp.Wt3 + (i / kC2) * kHid + (i % kC2) * 8);
    for (int i = tid; i < (kN3 - kOutPad) * kC2; i += kTile)
        *reinterpret_cast<uint4*>(sh.W3 + tc::canon_off(kOutPad + i / kC2, 8 * (i % kC2), kHid)) = make_uint4(0, 0, 0, 0);
    if (tid < kHid) { sh.b1[tid] = cp.b1[tid]; sh.b2[tid] = cp.b2[tid]; }
    if (tid < kOutPad) sh.b3[tid] = cp.b3[tid];
    if (tid < kIn) { sh.mean[tid] = cp.mean[tid]; sh.scale[tid] = cp.scale[tid]; }
    if (tid < kOut) sh.out_scale[tid] = cp.out_scale[tid];
    // one group with the first tile's gather: the first wait covers both
    if ((int)blockIdx.x < ntiles) closure_prefetch(sh, src, a, ntx, blockIdx.x, 0, tid, lane, ly);
    else cp_async_commit();
    if (ly == 0) tc::tmem_alloc<kTmemCols>(&sh.tmem);
    if (tid == 0) { tc::mbar_init(&sh.mbar[0], 1); tc::mbar_init(&sh.mbar[1], 1); }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sh.tmem;
    // this warp's 32 nodes are rows 32 (ly % 4) .. + 31 of M block ly / 4
    const int h = ly >> 2, hrow = tid & 127;
    const uint32_t tlane = tmem + 64 * h + ((uint32_t)(32 * (ly & 3)) << 16);
    uint32_t phase = 0;
    bool failed = false;
    int b = 0;
    for (int tl = blockIdx.x; tl < ntiles; tl += gridDim.x, b ^= 1) {
        const int next = tl + gridDim.x;
        // the other buffer's previous tile is done; parameters loaded; stop
        // everywhere once either M block has given up
        if (__syncthreads_or(failed)) { failed = true; break; }
        if (next < ntiles) closure_prefetch(sh, src, a, ntx, next, b ^ 1, tid, lane, ly);
        else cp_async_commit();  // empty group: keeps the wait count uniform
        cp_async_wait<1>();      // this tile's group has landed (for this thread)
        __syncthreads();         // ... and for every thread
        const int x0 = (tl % ntx) * kCTX, y0 = (tl / ntx) * kCTY;
        const int x = x0 + lane, y = y0 + ly;
        const bool inside = x < a.nx && y < a.ny;
        float f[9], g[10];
        if (tid < kHalo) {
            int hx, hy;
            ring_pos(tid, hx, hy);
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = sh.hpop[b][i][tid];
#pragma unroll
            for (int q = 0; q < 10; ++q) g[q] = sh.hpop[b][9 + q][tid];
            const Moments<float> m = moments(f, g, a.np.rho0);
            sh.mom[0][hy][hx] = m.ux; sh.mom[1][hy][hx] = m.uy;
            sh.mom[2][hy][hx] = m.bx; sh.mom[3][hy][hx] = m.by;
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = sh.pop[b][i][tid];
#pragma unroll
        for (int q = 0; q < 10; ++q) g[q] = sh.pop[b][9 + q][tid];
        float feat[kIn];
        point_features(f, g, a.np.rho0, feat);
        sh.mom[0][ly + 1][lane + 1] = feat[1]; sh.mom[1][ly + 1][lane + 1] = feat[2];
        sh.mom[2][ly + 1][lane + 1] = feat[3]; sh.mom[3][ly + 1][lane + 1] = feat[4];
        __syncthreads();
        stencil_features<kCHX, kCHY>(sh.mom, lane, ly, feat + 8);
        // normalised features, row hrow of M block h's K = 32 layer-1 operand
#pragma unroll
        for (int c = 0; c < kInPad; c += 8) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k0 = c + 2 * j, k1 = k0 + 1;
                const float v0 = (inside && k0 < kIn) ? (feat[k0] - sh.mean[k0]) * sh.scale[k0] : 0.f;
                const float v1 = (inside && k1 < kIn) ? (feat[k1] - sh.mean[k1]) * sh.scale[k1] : 0.f;
                w[j] = pack2(v0, v1);
            }
            *reinterpret_cast<uint4*>(sh.act[h] + tc::canon_off(hrow, c, kInPad)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        // three layers of this M block: operand writes -> async proxy, the
        // block's first thread issues, its 128 threads wait
        float out[kN3];
#pragma unroll 1
        for (int layer = 0; layer < 3; ++layer) {
            tc::fence_smem_to_async();
            tc::fence_before_sync();
            half_bar_or(h, false);
            tc::fence_after_sync();
            if (hrow == 0) {
                if (layer == 0) issue_layer<kInPad, kHid>(sh, h, sh.W1, tmem);
                else if (layer == 1) issue_layer<kHid, kHid>(sh, h, sh.W2, tmem);
                else issue_layer<kHid, kN3>(sh, h, sh.W3, tmem);
            }
            const bool ok = tc::mbar_wait(&sh.mbar[h], phase, kMbarWaitLimit);
            phase ^= 1;
            tc::fence_after_sync();
            if (half_bar_or(h, !ok)) {
                failed = true;
                break;
            }
            if (layer == 0) relu_to_act(sh, h, sh.b1, tlane, hrow);
            else if (layer == 1) relu_to_act(sh, h, sh.b2, tlane, hrow);
            else tc::ld16(tlane, out);
        }
        if (failed) continue;  // the next tile's first barrier stops both M blocks
        if (inside) {
            const float da[3] = {(out[0] + sh.b3[0]) * sh.out_scale[0], (out[1] + sh.b3[1]) * sh.out_scale[1],
                                 (out[2] + sh.b3[2]) * sh.out_scale[2]};
            if (cp.da_out) {
                const long long nn = (long long)a.nx * a.ny, node = (long long)y * a.nx + x;
#pragma unroll
                for (int k = 0; k < 3; ++k) cp.da_out[k * nn + node] = da[k];
            }
            collide_impl<true, float>(f, g, a.np, da);
            const long long o = (long long)y * a.pitch + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) dst[(long long)i * a.plane + o] = f[i];
#pragma unroll
            for (int q = 0; q < 10; ++q) dst[(long long)(9 + q) * a.plane + o] = g[q];
        }
    }
    // every thread arrives here; one M block may have given up on its last tile
    if (__syncthreads_or(failed)) {
        if (tid == 0) atomicExch(cp.err, 1);
        // the MMAs may still be running: wait for them (bounded) before the
        // tensor memory is given back
        tc::mbar_wait(&sh.mbar[h], phase ^ 1, kMbarWaitLimit);
    }
    cp_async_wait<0>();  // nothing left in flight when the block exits
    tc::fence_before_sync();
    __syncthreads();
    if (ly == 0) tc::tmem_free<kTmemCols>(tmem);
}

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
    const int ntx = (s.L.nx + kCTX - 1) / kCTX, nty = (s.L.ny + kCTY - 1) / kCTY, ntiles = ntx * nty;
    const size_t smem = sizeof(ClosureSharedTC);
    cudaError_t e = cudaFuncSetAttribute(step_closure_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // all of the unified L1 / shared storage as shared memory, so that two
    // blocks fit on an SM (the default carve-out leaves room for one)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_closure_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0, dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_closure_tc, 256, smem);
    if (e != cudaSuccess) return e;
    // The occupancy calculator answers one block per SM for this kernel (it
    // allocates tensor memory); registers (launch bounds) and shared memory
    // (static_assert) fit two, and two blocks hold 2 x 128 of the 512 columns.
    const int blocks = std::max(1, std::min(ntiles, std::max(2, per_sm) * sms));
    step_closure_tc<<<blocks, dim3(kCTX, kCTY), smem, st>>>(a, cp, ntx, ntiles);
    return cudaGetLastError();
}

}  // namespace mhd
