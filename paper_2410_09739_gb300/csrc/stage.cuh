// stage.cuh -- row-staged variant of the paired step kernel (launch variant 3).
//
// One tile is one x-row of the box (fixed y, z), all 27 slots.  A persistent
// CTA walks the rows t = blockIdx.x + k gridDim.x through a ring of ns
// shared-memory stages, each holding the 27 slot rows of one tile:
//
//   load   one elected thread moves the 27 source rows of a tile into a
//          stage with bulk asynchronous copies (cp.async.bulk, completion
//          counted in bytes on the stage's mbarrier).  Even step: the cell's
//          own slot rows.  Odd step: for slot s the row (y - e_y, z - e_z) of
//          slot 26 - s, i.e. the row the populations stream in from (Step 6);
//          where that row lies in a wall (half-way bounce-back at y = -1/2 or
//          ny - 1/2) the tile's own row of slot s, which holds the reflected
//          value the even step parked there (the AA pattern of cell.cuh).
//   compute  every thread takes two neighbouring cells x, x + 1 of the row,
//          reads its 27 value pairs from the stage (the x - e_x shift and the
//          periodic x wrap are shared-memory indices), collides them with the
//          packed fp32 arithmetic of pair.cuh (the same collide_cell as the
//          paired kernel, so the results are bit-identical to it), and writes
//          each post-collision value back into the stage at its streamed
//          position x + e_x (odd step; the cell itself where the link meets a
//          wall) or in place (even step);
//   store  the elected thread bulk-stores the 27 rows to their destination
//          rows: even step the tile's own row of slot 26 - s; odd step the row
//          (y + e_y, z + e_z) of slot s, or the tile's own row of slot 26 - s
//          for a link into a wall.
//
// The AA pattern makes this race-free: within one step the rows a tile reads
// are exactly the rows it writes, and no other tile touches them.  A stage is
// reloaded only after the bulk store that reads it has finished reading
// (cp.async.bulk.wait_group.read).  While a tile is computed the loads of the
// next ns - 2 tiles are in flight.
//
// Requirements (checked by the host): periodic box or y walls; nx * sizeof(S)
// a multiple of 16 (bulk copies move 16-byte multiples between 16-byte-aligned
// addresses; slot rows start 128-byte aligned); nx <= 2 * 512.
//
// Every wait is bounded: a stage whose data has not arrived after about a
// second makes the CTA set bit 2 of the flag, wait (again bounded) for its
// copies in flight, and return without storing; the host then reports
// FPCLBM_ERR_TIMEOUT.
#pragma once
#include "cell.cuh"
#include "internal.h"

namespace fpc {

constexpr int kStageMaxThreads = 512;

inline StepArgs<f2> pair_args(const StepArgs<float>& a);  // step_kernel.cuh
constexpr int kStageFlagTimeout = 2;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Wait for the phase of parity `parity` of an mbarrier to complete; false after ~1 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void bulk_store(void* dst, uint32_t src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(src), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// all but the most recent bulk-store group have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all_but_last() { asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory"); }
// every bulk-store group has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// shared-memory writes of this thread become visible to the bulk copies (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Pair access to a stage: two values of one slot row at indices i, j (as f2 lanes x, y).
template <typename S>
__device__ __forceinline__ f2 stage_ld(const S* row, unsigned i, unsigned j)
{
    return f2(Store<S>::ld(row + i), Store<S>::ld(row + j));
}
template <typename S>
__device__ __forceinline__ void stage_st(S* row, unsigned i, unsigned j, f2 v)
{
    Store<S>::st(row + i, v.v.x);
    Store<S>::st(row + j, v.v.y);
}

// One bulk copy of `rows` consecutive slot rows between global memory and stage chunk row `lr`.
struct RowSpan {
    int slot, y, z, rows, lr;  // global slot, first row y of plane z, row count, first local row
};

// Where the rows of stage chunk s come from (load) or go to (store), for the tile of rows
// y0 .. y0 + R - 1 of plane z: one span, or two where the tile touches the periodic y wrap or a
// y wall.  Load: local row r holds what streams into row y0 + r, i.e. row y0 + r - e_y of slot
// 26 - s (odd step), or the own row of slot s where that row lies in a wall; even step the own
// rows of slot s.  Store: local row r goes to row y0 + r + e_y of slot s (odd step), or to the
// own row of slot 26 - s for a link into a wall; even step the own rows of slot 26 - s.
template <bool ODD, int BC>
__device__ __forceinline__ int stage_spans(bool store, int s, int y0, int z, int R, int ny, int nz, RowSpan (&sp)[2])
{
    if (!ODD) {
        sp[0] = {store ? 26 - s : s, y0, z, R, 0};
        return 1;
    }
    const int ey = (s / 3) % 3 - 1, ez = s / 9 - 1;
    const int dy = store ? ey : -ey, dz = store ? ez : -ez;  // neighbour offset of the moved rows
    int zn = z + dz;
    zn = zn < 0 ? nz - 1 : (zn == nz ? 0 : zn);
    const int sn = store ? s : 26 - s;  // slot of the neighbour rows
    const int sw = store ? 26 - s : s;  // slot of the own row at a wall
    if (dy == 0 || (y0 + dy >= 0 && y0 + R - 1 + dy < ny)) {
        sp[0] = {sn, y0 + dy, zn, R, 0};
        return 1;
    }
    // dy = -1: local row 0 (y0 = 0) crosses y = -1; local rows 1 .. R-1 take rows y0 .. y0+R-2.
    // dy = +1: local row R-1 (y0+R-1 = ny-1) crosses y = ny; local rows 0 .. R-2 take rows y0+1 .. y0+R-1.
    int n = 0, edge;
    if (dy < 0) {
        edge = 0;
        if (R > 1) sp[n++] = {sn, y0, zn, R - 1, 1};
    } else {
        edge = R - 1;
        if (R > 1) sp[n++] = {sn, y0 + 1, zn, R - 1, 0};
    }
    if (BC == BC_WALLS_Y)  // the crossing row's own row of the wall slot, same plane
        sp[n++] = {sw, y0 + edge, z, 1, edge};
    else  // periodic wrap in y
        sp[n++] = {sn, dy < 0 ? ny - 1 : 0, zn, 1, edge};
    return n;
}

// CB: bytes of one slot chunk of a stage (a compile-time constant, so that every shared-memory
// access of the compute phase is an immediate offset); a tile holds R whole rows, R nx <= CB /
// sizeof(S).
template <typename S, bool ODD, int BC, bool FORCE, int MODE, int CB>
__global__ void __launch_bounds__(kStageMaxThreads) k_step_stage(const StepArgs<f2> a, const FastDiv div_tpp,
                                                                 const unsigned ntiles, const int ns, const int R)
{
    static_assert(BC == BC_PERIODIC || BC == BC_WALLS_Y, "periodic box or y walls");
    constexpr bool WALLS = BC == BC_WALLS_Y;
    constexpr int TC = CB / (int)sizeof(S);  // entries per slot chunk
    constexpr unsigned stageb = 27u * CB;
    extern __shared__ __align__(128) unsigned char stage_smem[];
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const unsigned rowb = (unsigned)nx * sizeof(S);
    const unsigned tpp = (unsigned)(ny / R);  // tiles per plane
    const uint32_t sm0 = smem_addr(stage_smem);
    const uint32_t bar0 = sm0 + (unsigned)ns * stageb;  // ns mbarriers of 8 bytes after the stages
    const unsigned tid = threadIdx.x, lane = tid & 31u;
    const bool producer = tid < 27;  // lane s of warp 0 moves slot s
    unsigned char* const gbuf = static_cast<unsigned char*>(a.buf);
    const size_t slotb = (size_t)a.stride * sizeof(S);

    if (tid == 0) {
        for (int k = 0; k < ns; ++k) mbar_init(bar0 + 8u * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        fence_proxy_async_smem();
    }
    __syncthreads();

    auto tile_yz = [&](unsigned t, int& y0, int& z) {
        z = (int)fdiv(t, div_tpp);
        y0 = (int)(t - (unsigned)z * tpp) * R;
    };
    auto gaddr = [&](const RowSpan& q) {
        return gbuf + (size_t)q.slot * slotb + (size_t)((unsigned)q.y + (unsigned)ny * (unsigned)q.z) * rowb;
    };
    // warp 0: lane 0 arms the stage's barrier, lanes 0..26 load their slot's rows
    auto issue_load = [&](unsigned t, int k) {
        int y0, z;
        tile_yz(t, y0, z);
        const uint32_t bar = bar0 + 8u * k;
        if (lane == 0) mbar_arrive_expect_tx(bar, 27u * (unsigned)R * rowb);
        __syncwarp();
        if (producer) {
            RowSpan sp[2];
            const int n = stage_spans<ODD, BC>(false, (int)tid, y0, z, R, ny, nz, sp);
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (q < n)
                    bulk_load(sm0 + (unsigned)k * stageb + tid * (unsigned)CB + (unsigned)sp[q].lr * rowb, gaddr(sp[q]),
                              (unsigned)sp[q].rows * rowb, bar);
        }
    };
    auto issue_store = [&](unsigned t, int k) {
        int y0, z;
        tile_yz(t, y0, z);
        if (producer) {
            RowSpan sp[2];
            const int n = stage_spans<ODD, BC>(true, (int)tid, y0, z, R, ny, nz, sp);
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (q < n)
                    bulk_store(gaddr(sp[q]), sm0 + (unsigned)k * stageb + tid * (unsigned)CB + (unsigned)sp[q].lr * rowb,
                               (unsigned)sp[q].rows * rowb);
            bulk_commit();
        }
    };

    // prologue: the first ns - 1 tiles of this CTA in flight
    unsigned pending = 0;  // stages with loads in flight (warp 0)
    if (tid < 32)
        for (int k = 0; k < ns - 1; ++k) {
            const unsigned t = blockIdx.x + (unsigned)k * gridDim.x;
            if (t < ntiles) {
                issue_load(t, k);
                pending |= 1u << k;
            }
        }

    // this thread's cells x, x + 1 of local row r and their wrapped neighbours in the row
    const unsigned half = (unsigned)nx / 2;
    const unsigned r = tid / half, x = 2u * (tid - r * half);
    const bool act = r < (unsigned)R;
    const unsigned rb = r * (unsigned)nx;
    const unsigned ia = rb + x;                                    // the cells' own entries
    const unsigned im1 = rb + (x == 0 ? (unsigned)nx - 1 : x - 1);  // x - 1 of the first cell
    const unsigned ip2 = rb + (x + 2 == (unsigned)nx ? 0u : x + 2); // x + 1 of the second cell
    const Rates<f2>& rt = a.rates;
    unsigned parity = 0;  // bit k: phase parity of stage k's next completion
    bool timed_out = false;
    int k = 0;
    for (unsigned t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const bool ok = mbar_wait_bounded(bar0 + 8u * k, (parity >> k) & 1u);
        S* const st = reinterpret_cast<S*>(stage_smem + (size_t)k * stageb);
        bool top = false, bot = false;  // this thread's row touches the wall y = ny - 1/2 / y = -1/2
        if (WALLS) {
            const unsigned y = (t - fdiv(t, div_tpp) * tpp) * (unsigned)R + r;
            bot = y == 0;
            top = y + 1 == (unsigned)ny;
        }
        f2 g[27];
        if (ok && act) {
#pragma unroll
            for (int s = 0; s < 27; ++s) {
                const S* row = st + s * TC;
                const int ix = s % 3, iy = (s / 3) % 3;
                // the value streaming in for slot s comes from x - e_x (e_x = ix - 1); a source in the
                // wall is the cell's own reflected value (no shift)
                const bool wall = WALLS && ((iy == 2 && bot) || (iy == 0 && top));
                if (!ODD || ix == 1) {
                    g[s] = Store2<S>::ld(row + ia);
                } else if (ix == 0) {  // e_x = -1: sources x + 1, x + 2
                    g[s] = wall ? Store2<S>::ld(row + ia) : stage_ld(row, ia + 1, ip2);
                } else {  // e_x = +1: sources x - 1, x
                    g[s] = wall ? Store2<S>::ld(row + ia) : stage_ld(row, im1, ia);
                }
            }
        }
        // odd step: a thread's writes land on its neighbours' read positions
        if (ODD) __syncthreads();
        if (ok && act) {
            const bool fine = collide_cell<f2, FORCE, MODE>(g, rt, a.Fx, a.Fy, a.Fz, rt.om[4], rt.om[5], rt.om[6],
                                                            rt.om[8], rt.om[9], nullptr);
            if (!fine) atomicOr(a.flag, 1);
#pragma unroll
            for (int s = 0; s < 27; ++s) {
                S* row = st + s * TC;
                const int ix = s % 3, iy = (s / 3) % 3;
                // destination x + e_x; a link into the wall stays at the cell (reflected)
                const bool wall = WALLS && ((iy == 0 && bot) || (iy == 2 && top));
                if (!ODD || ix == 1) {
                    Store2<S>::st(row + ia, g[s]);
                } else if (ix == 2) {  // e_x = +1: destinations x + 1, x + 2
                    if (wall) Store2<S>::st(row + ia, g[s]);
                    else stage_st(row, ia + 1, ip2, g[s]);
                } else {  // e_x = -1: destinations x - 1, x
                    if (wall) Store2<S>::st(row + ia, g[s]);
                    else stage_st(row, im1, ia, g[s]);
                }
            }
        }
        fence_proxy_async_smem();
        if (__syncthreads_or(!ok)) {  // some thread's stage never arrived: stop, store nothing
            timed_out = true;
            break;
        }
        parity ^= 1u << k;
        if (tid < 32) {
            pending &= ~(1u << k);
            issue_store(t, k);
            // the stage of the previous tile is free once its store has read it (each lane waits
            // for its own slot's store): refill it with the tile ns - 1 ahead of this one
            const int kp = k == 0 ? ns - 1 : k - 1;
            const unsigned tn = t + (unsigned)(ns - 1) * gridDim.x;
            if (tn < ntiles) {
                if (producer) bulk_wait_read_all_but_last();
                issue_load(tn, kp);
                pending |= 1u << kp;
            }
        }
        k = k + 1 == ns ? 0 : k + 1;
    }
    if (tid < 32) {
        if (timed_out && tid == 0) {
            atomicOr(a.flag, kStageFlagTimeout);
            // let the copies still in flight land before the CTA's shared memory is released
            for (int q = 0; q < ns; ++q)
                if (pending & (1u << q)) mbar_wait_bounded(bar0 + 8u * q, (parity >> q) & 1u);
        }
        if (producer) bulk_wait_all();
    }
}

// Rows per tile: the largest R with R nx <= entries of a chunk that divides ny (1 if none).
inline int stage_rows(int nx, int ny, int chunk_entries)
{
    for (int R = chunk_entries / nx; R > 1; --R)
        if (ny % R == 0) return R;
    return 1;
}

// Launch: one CTA per resident slot (persistent), R nx / 2 threads rounded up to a warp, ns stages.
template <typename S, bool ODD, int BC, bool FORCE, int MODE, int CB>
cudaError_t step_go_stage_cb(const StepArgs<float>& a, int ns, cudaStream_t st)
{
    constexpr int TC = CB / (int)sizeof(S);
    const int R = stage_rows(a.nx, a.ny, TC);
    const int threads = (R * a.nx / 2 + 31) / 32 * 32;
    const size_t smem = (size_t)ns * 27 * CB + 8 * (size_t)ns;
    auto kern = k_step_stage<S, ODD, BC, FORCE, MODE, CB>;
    // resident blocks per SM for the last (threads, shared memory) this instantiation launched with,
    // on the device of that launch (a benign race: every thread computes the same values)
    static int c_dev = -1, c_threads = 0, c_per_sm = 0, c_sms = 0;
    static size_t c_smem = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    if (dev == c_dev && threads == c_threads && smem == c_smem) {
        per_sm = c_per_sm;
        sms = c_sms;
    } else {
        int optin = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        if (smem > (size_t)optin) return cudaErrorInvalidValue;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        c_per_sm = per_sm;
        c_sms = sms;
        c_threads = threads;
        c_smem = smem;
        c_dev = dev;
    }
    const unsigned ntiles = (unsigned)(a.ny / R) * (unsigned)a.nz;
    unsigned grid = (unsigned)(per_sm * sms);
    if (grid > ntiles) grid = ntiles;
    kern<<<grid, threads, smem, st>>>(pair_args(a), make_fastdiv((unsigned)(a.ny / R)), ntiles, ns, R);
    return cudaGetLastError();
}

// Chunks of 1 KB (rows up to 1 KB: 512 cells of 16-bit storage, 256 of fp32) or 2 KB.
template <typename S, bool ODD, int BC, bool FORCE, int MODE>
cudaError_t step_go_stage(const StepArgs<float>& a, int ns, cudaStream_t st)
{
    const size_t rowb = (size_t)a.nx * sizeof(S);
    if (rowb % 16 != 0 || rowb > 2048 || a.nx < 2 || ns < 3 || ns > 8) return cudaErrorInvalidValue;
    if (rowb <= 1024) return step_go_stage_cb<S, ODD, BC, FORCE, MODE, 1024>(a, ns, st);
    return step_go_stage_cb<S, ODD, BC, FORCE, MODE, 2048>(a, ns, st);
}

}  // namespace fpc
