// stage.cuh -- row-staged variant of the paired step kernel (launch variant 3).
//
// A tile is R whole x-rows of the box (rows y0 .. y0+R-1 of one plane z, all
// 27 slots).  Each CTA is a warp-specialised pipeline over the tiles
// t = blockIdx.x + k gridDim.x:
//
//   producer warp   lane s (s < 27) moves slot s: bulk asynchronous copies
//                   (cp.async.bulk) of the tile's source rows into an input
//                   stage, completion counted in bytes on the stage's "full"
//                   mbarrier, and, once the consumers have filled an output
//                   stage, bulk copies of its rows to their destinations.
//                   Even step: the cells' own rows of slot s in, of slot
//                   26 - s out.  Odd step: in, the rows y - e_y of slot 26 - s
//                   (where the populations stream from, Step 6), or the own row
//                   of slot s where that row lies in a y wall; out, the rows
//                   y + e_y of slot s, or the own row of slot 26 - s for a link
//                   into a wall (half-way bounce-back, the AA pattern of
//                   cell.cuh).  Periodic wrap in y and z.
//   consumer warps  every thread takes two neighbouring cells x, x + 1 of a
//                   row, reads its 27 value pairs from the input stage (the
//                   x - e_x shift and the periodic x wrap are shared-memory
//                   indices), releases the stage, collides the pair with the
//                   packed fp32 arithmetic of pair.cuh (the same collide_cell
//                   as the paired kernel: results bit-identical to it), and
//                   writes each post-collision value into the output stage at
//                   its streamed position x + e_x (odd step; the cell itself
//                   for a link into a wall) or in place (even step).
//
// Handshakes (no block-wide barrier after set-up): full_in (producer -> the
// consumers: data arrived), empty_in (consumers -> producer: stage read),
// full_out (consumers -> producer: output written), empty_out (producer ->
// consumers: the bulk store has read the output stage).  The AA pattern makes
// the in-place update race-free across tiles: within one step the rows a tile
// reads are exactly the rows it writes, and no other tile touches them.
//
// Requirements (checked by the host): periodic box or y walls; nx * sizeof(S)
// a multiple of 16 (bulk copies move 16-byte multiples between 16-byte-aligned
// addresses; slot rows start 128-byte aligned); nx at most the tile capacity.
//
// Every wait is bounded: after about a second a waiting thread sets a shared
// abort word, which ends every other wait of the CTA at once; the producer
// then waits (bounded) for its copies in flight, nothing more is stored, and
// the CTA sets bit 2 of the flag (the host reports FPCLBM_ERR_TIMEOUT).
#pragma once
#include "cell.cuh"
#include "internal.h"

namespace fpc {

inline StepArgs<f2> pair_args(const StepArgs<float>& a);  // step_kernel.cuh
constexpr int kStageFlagTimeout = 2;
constexpr unsigned kStageOut = 2;  // output stages (a power of two: stage and phase by shifts)

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

// Shared-memory access by 32-bit shared addresses (explicit ld.shared / st.shared).
__device__ __forceinline__ uint32_t lds32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.b32 %0, [%1];\n" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t lds16(uint32_t a)
{
    unsigned short v;
    asm volatile("ld.shared.b16 %0, [%1];\n" : "=h"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.b32 [%0], %1;\n" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts16(uint32_t a, unsigned short v)
{
    asm volatile("st.shared.b16 [%0], %1;\n" ::"r"(a), "h"(v) : "memory");
}
__device__ __forceinline__ f2 lds_f2(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return f2(v);
}
__device__ __forceinline__ void sts_f2(uint32_t a, f2 v)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(v.v.x), "f"(v.v.y) : "memory");
}

// Values of the storage type in a stage, converted exactly as Store / Store2 do (so the staged
// kernel stays bit-identical to the paired one): one entry, or two neighbouring entries (4- or
// 8-byte aligned) as the lanes of an f2.
template <typename S>
struct StageIO;
template <>
struct StageIO<float> {
    __device__ __forceinline__ static float ld1(uint32_t a) { return __uint_as_float(lds32(a)); }
    __device__ __forceinline__ static f2 ld2(uint32_t a) { return lds_f2(a); }
    __device__ __forceinline__ static void st1(uint32_t a, float v) { sts32(a, __float_as_uint(v)); }
    __device__ __forceinline__ static void st2(uint32_t a, f2 v) { sts_f2(a, v); }
};
template <>
struct StageIO<__nv_bfloat16> {
    __device__ __forceinline__ static float ld1(uint32_t a) { return __uint_as_float(lds16(a) << 16); }
    __device__ __forceinline__ static f2 ld2(uint32_t a)
    {
        const uint32_t w = lds32(a);
        return f2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    __device__ __forceinline__ static void st1(uint32_t a, float v)
    {
        sts16(a, __bfloat16_as_ushort(__float2bfloat16_rn(v)));
    }
    __device__ __forceinline__ static void st2(uint32_t a, f2 v)
    {
        const __nv_bfloat162 b = __float22bfloat162_rn(v.v);
        sts32(a, *reinterpret_cast<const uint32_t*>(&b));
    }
};
template <>
struct StageIO<__half> {
    __device__ __forceinline__ static float ld1(uint32_t a) { return __half2float(__ushort_as_half((unsigned short)lds16(a))); }
    __device__ __forceinline__ static f2 ld2(uint32_t a)
    {
        const uint32_t w = lds32(a);
        return f2(__half22float2(*reinterpret_cast<const __half2*>(&w)));
    }
    __device__ __forceinline__ static void st1(uint32_t a, float v) { sts16(a, __half_as_ushort(__float2half_rn(v))); }
    __device__ __forceinline__ static void st2(uint32_t a, f2 v)
    {
        const __half2 h = __float22half2_rn(v.v);
        sts32(a, *reinterpret_cast<const uint32_t*>(&h));
    }
};

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

// The 27 value pairs of cells x, x + 1 in a stage (byte addresses of slot chunk 0: pa the cells'
// own entries, pm1 entry x - 1, pp2 entry x + 2, all in the same row).  Odd step: the value
// streaming in for slot s comes from x - e_x (e_x = ix - 1); a source in a y wall is the cell's own
// reflected value (no shift).  Even step: the own entries.
template <typename S, bool ODD, bool WALLS, unsigned CB>
__device__ __forceinline__ void stage_read(f2 (&g)[27], uint32_t pa, uint32_t pm1, uint32_t pp2, bool bot, bool top)
{
    constexpr unsigned ES = sizeof(S);
#pragma unroll
    for (int s = 0; s < 27; ++s) {
        const unsigned so = (unsigned)s * CB;  // slot chunk offset (compile-time)
        const int ix = s % 3, iy = (s / 3) % 3;
        const bool wall = WALLS && ((iy == 2 && bot) || (iy == 0 && top));
        if (!ODD || ix == 1) {
            g[s] = StageIO<S>::ld2(pa + so);
        } else if (ix == 0) {  // e_x = -1: sources x + 1, x + 2
            g[s] = wall ? StageIO<S>::ld2(pa + so) : f2(StageIO<S>::ld1(pa + so + ES), StageIO<S>::ld1(pp2 + so));
        } else {  // e_x = +1: sources x - 1, x
            g[s] = wall ? StageIO<S>::ld2(pa + so) : f2(StageIO<S>::ld1(pm1 + so), StageIO<S>::ld1(pa + so));
        }
    }
}

// The post-collision pairs of cells x, x + 1 into a stage: odd step at the streamed position
// x + e_x (the cell itself for a link into a y wall, reflected), even step in place.  Over all
// threads of a row every entry is written once.
template <typename S, bool ODD, bool WALLS, unsigned CB>
__device__ __forceinline__ void stage_write(const f2 (&g)[27], uint32_t qa, uint32_t qm1, uint32_t qp2, bool bot,
                                            bool top)
{
    constexpr unsigned ES = sizeof(S);
#pragma unroll
    for (int s = 0; s < 27; ++s) {
        const unsigned so = (unsigned)s * CB;
        const int ix = s % 3, iy = (s / 3) % 3;
        const bool wall = WALLS && ((iy == 0 && bot) || (iy == 2 && top));
        if (!ODD || ix == 1) {
            StageIO<S>::st2(qa + so, g[s]);
        } else if (ix == 2) {  // e_x = +1: destinations x + 1, x + 2
            if (wall) {
                StageIO<S>::st2(qa + so, g[s]);
            } else {
                StageIO<S>::st1(qa + so + ES, g[s].v.x);
                StageIO<S>::st1(qp2 + so, g[s].v.y);
            }
        } else {  // e_x = -1: destinations x - 1, x
            if (wall) {
                StageIO<S>::st2(qa + so, g[s]);
            } else {
                StageIO<S>::st1(qm1 + so, g[s].v.x);
                StageIO<S>::st1(qa + so, g[s].v.y);
            }
        }
    }
}

// Bounded wait on an mbarrier phase that also gives up when another thread of the CTA has
// aborted; a wait that runs out (about a second) aborts the CTA.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (global_ns() - t0 > 1000000000ull) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// Resident blocks per SM the registers are capped for: four blocks of 4 consumer warps (96
// registers) for the unit-rate collision without force, which fits them without spilling, three
// for the other modes; two blocks of 6 consumer warps (146 registers); one block of 8.
__host__ __device__ constexpr int stage_min_blocks(int NCW, bool FORCE, int MODE)
{
    return NCW == 4 ? ((r1_mode(MODE) && !FORCE) ? 4 : 3) : NCW == 6 ? 2 : 1;
}

// NCW consumer warps (two cells per thread: tiles of up to 64 NCW cells) and one producer warp.
// CB, the bytes of one slot chunk of a stage, is a compile-time constant, so that every
// shared-memory access of the compute phase is an immediate offset; a tile holds R whole rows,
// R nx <= CB / sizeof(S).
template <typename S, bool ODD, int BC, bool FORCE, int MODE, int NCW>
__global__ void __launch_bounds__(32 * (NCW + 1), stage_min_blocks(NCW, FORCE, MODE)) k_step_stage(const StepArgs<f2> a, const FastDiv div_tpp,
                                                               const unsigned ntiles, const int R, const int nsi)
{
    static_assert(BC == BC_PERIODIC || BC == BC_WALLS_Y, "periodic box or y walls");
    constexpr bool WALLS = BC == BC_WALLS_Y;
    constexpr unsigned NC = 32 * NCW;            // consumer threads
    constexpr int TC = 2 * (int)NC;              // entries per slot chunk (cells per tile at most)
    constexpr unsigned CB = TC * sizeof(S);      // bytes per slot chunk
    constexpr unsigned STB = 27u * CB;           // bytes per stage
    constexpr unsigned nso = kStageOut;          // output stages
    extern __shared__ __align__(128) unsigned char stage_smem[];
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const unsigned rowb = (unsigned)nx * sizeof(S);
    const unsigned tpp = (unsigned)(ny / R);  // tiles per plane
    const uint32_t sm0 = smem_addr(stage_smem);
    const uint32_t in0 = sm0, out0 = sm0 + (unsigned)nsi * STB;
    const uint32_t bars = out0 + (unsigned)nso * STB;
    const uint32_t full_in = bars, empty_in = bars + 8u * nsi, full_out = bars + 16u * nsi,
                   empty_out = bars + 16u * nsi + 8u * nso;
    volatile int* abort = reinterpret_cast<volatile int*>(stage_smem + (bars - sm0) + 16u * (nsi + nso));
    const unsigned tid = threadIdx.x, lane = tid & 31u;
    unsigned char* const gbuf = static_cast<unsigned char*>(a.buf);
    const size_t slotb = (size_t)a.stride * sizeof(S);

    if (tid == 0) {
        for (int k = 0; k < nsi; ++k) {
            mbar_init(full_in + 8u * k, 1);
            mbar_init(empty_in + 8u * k, NC);
        }
        for (int j = 0; j < nso; ++j) {
            mbar_init(full_out + 8u * j, NC);
            mbar_init(empty_out + 8u * j, 1);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        fence_proxy_async_smem();
    }
    __syncthreads();

    // this CTA's tiles: t_i = blockIdx.x + i gridDim.x, i < nt
    const unsigned nt = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (tid >= NC) {  // ---------------- producer warp ----------------
        const bool mover = lane < 27;  // lane s moves slot s
        auto tile_yz = [&](unsigned i, int& y0, int& z) {
            const unsigned t = blockIdx.x + i * gridDim.x;
            z = (int)fdiv(t, div_tpp);
            y0 = (int)(t - (unsigned)z * tpp) * R;
        };
        auto gaddr = [&](const RowSpan& q) {
            return gbuf + (size_t)q.slot * slotb + (size_t)((unsigned)q.y + (unsigned)ny * (unsigned)q.z) * rowb;
        };
        auto issue_load = [&](unsigned i, int k) {
            int y0, z;
            tile_yz(i, y0, z);
            const uint32_t bar = full_in + 8u * k;
            if (lane == 0) mbar_arrive_expect_tx(bar, 27u * (unsigned)R * rowb);
            __syncwarp();
            if (mover) {
                RowSpan sp[2];
                const int n = stage_spans<ODD, BC>(false, (int)lane, y0, z, R, ny, nz, sp);
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    if (q < n)
                        bulk_load(in0 + (unsigned)k * STB + lane * CB + (unsigned)sp[q].lr * rowb, gaddr(sp[q]),
                                  (unsigned)sp[q].rows * rowb, bar);
            }
        };
        auto issue_store = [&](unsigned i, int j) {
            int y0, z;
            tile_yz(i, y0, z);
            if (mover) {
                RowSpan sp[2];
                const int n = stage_spans<ODD, BC>(true, (int)lane, y0, z, R, ny, nz, sp);
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    if (q < n)
                        bulk_store(gaddr(sp[q]), out0 + (unsigned)j * STB + lane * CB + (unsigned)sp[q].lr * rowb,
                                   (unsigned)sp[q].rows * rowb);
                bulk_commit();
            }
        };
        unsigned lastpar = 0;  // bit k: parity of the phase of the last load issued into input stage k
        unsigned issued = 0;   // bit k: input stage k has received a load
        const unsigned pro = nt < (unsigned)nsi ? nt : (unsigned)nsi;
        for (unsigned k = 0; k < pro; ++k) {
            issue_load(k, (int)k);
            issued |= 1u << k;
        }
        bool ok = true;
        int ki = 0;
        unsigned pin = 0;  // (i / nsi) & 1, kept without dividing
        for (unsigned i = 0; i < nt; ++i) {
            const unsigned ko = i % nso, pout = (i / nso) & 1u;
            // refill input stage ki with tile i + nsi once the consumers have read tile i from it
            if (i + nsi < nt) {
                ok = mbar_wait_or_abort(empty_in + 8u * ki, pin, abort);
                if (!ok) break;
                issue_load(i + nsi, ki);
                lastpar ^= 1u << ki;
            }
            // store tile i once the consumers have written it
            ok = mbar_wait_or_abort(full_out + 8u * ko, pout, abort);
            if (!ok) break;
            issue_store(i, ko);
            // the previous tile's output stage is free once its store has read it
            if (i >= 1) {
                if (mover) bulk_wait_read_all_but_last();
                __syncwarp();
                if (lane == 0) mbar_arrive(empty_out + 8u * (ko == 0 ? nso - 1 : ko - 1));
            }
            if (++ki == nsi) {
                ki = 0;
                pin ^= 1u;
            }
        }
        if (!ok && lane == 0) {
            atomicOr(a.flag, kStageFlagTimeout);
            // let the loads still in flight land before the CTA's shared memory is released
            for (int k = 0; k < nsi; ++k)
                if (issued & (1u << k)) mbar_wait_bounded(full_in + 8u * k, (lastpar >> k) & 1u);
        }
        if (mover) bulk_wait_all();
        return;
    }

    // ---------------- consumer warps: cells x, x + 1 of local row r ----------------
    const unsigned half = (unsigned)nx / 2;
    const unsigned r = tid / half, x = 2u * (tid - r * half);
    const bool act = r < (unsigned)R;
    const unsigned rb = r * (unsigned)nx;
    const unsigned ia = rb + x;                                     // the cells' own entries
    const unsigned im1 = rb + (x == 0 ? (unsigned)nx - 1 : x - 1);  // x - 1 of the first cell
    const unsigned ip2 = rb + (x + 2 == (unsigned)nx ? 0u : x + 2); // x + 1 of the second cell
    const Rates<f2>& rt = a.rates;
    int ki = 0;
    unsigned pin = 0;  // (i / nsi) & 1, kept without dividing
    for (unsigned i = 0; i < nt; ++i) {
        const unsigned ko = i % nso, pout = (i / nso) & 1u;
        if (!mbar_wait_or_abort(full_in + 8u * ki, pin, abort)) return;
        bool top = false, bot = false;  // this thread's row touches the wall y = ny - 1/2 / y = -1/2
        if (WALLS) {
            const unsigned t = blockIdx.x + i * gridDim.x;
            const unsigned y = (t - fdiv(t, div_tpp) * tpp) * (unsigned)R + r;
            bot = y == 0;
            top = y + 1 == (unsigned)ny;
        }
        // byte addresses in this input stage of the cells' own entries and of their x neighbours
        constexpr unsigned ES = sizeof(S);
        const uint32_t ain = in0 + (unsigned)ki * STB;
        const uint32_t pa = ain + ES * ia, pm1 = ain + ES * im1, pp2 = ain + ES * ip2;
        f2 g[27];
        if (act) stage_read<S, ODD, WALLS, CB>(g, pa, pm1, pp2, bot, top);
        mbar_arrive(empty_in + 8u * ki);
        bool fine = true;
        if (act)
            fine = collide_cell<f2, FORCE, MODE>(g, rt, a.Fx, a.Fy, a.Fz, rt.om[4], rt.om[5], rt.om[6], rt.om[8],
                                                 rt.om[9], nullptr);
        if (!fine) atomicOr(a.flag, 1);
        if (i >= (unsigned)nso && !mbar_wait_or_abort(empty_out + 8u * ko, pout ^ 1u, abort)) return;
        const uint32_t aout = out0 + (unsigned)ko * STB;
        const uint32_t qa = aout + ES * ia, qm1 = aout + ES * im1, qp2 = aout + ES * ip2;
        if (act) stage_write<S, ODD, WALLS, CB>(g, qa, qm1, qp2, bot, top);
        fence_proxy_async_smem();
        mbar_arrive(full_out + 8u * ko);
        if (++ki == nsi) {
            ki = 0;
            pin ^= 1u;
        }
    }
}

// Rows per tile: the largest R with R nx <= the tile capacity that divides ny (1 if none).
inline int stage_rows(int nx, int ny, int cap)
{
    for (int R = cap / nx; R > 1; --R)
        if (ny % R == 0) return R;
    return 1;
}

// Launch: one CTA per resident slot (persistent); nsi input and kStageOut output stages.
template <typename S, bool ODD, int BC, bool FORCE, int MODE, int NCW>
cudaError_t step_go_stage_ncw(const StepArgs<float>& a, int nsi, cudaStream_t st)
{
    constexpr int TC = 64 * NCW;
    constexpr int nso = kStageOut;
    const int R = stage_rows(a.nx, a.ny, TC);
    const int threads = 32 * (NCW + 1);
    const size_t smem = (size_t)(nsi + nso) * 27 * TC * sizeof(S) + 16 * (size_t)(nsi + nso) + 16;
    auto kern = k_step_stage<S, ODD, BC, FORCE, MODE, NCW>;
    // resident blocks per SM for the last shared-memory size this instantiation launched with,
    // on the device of that launch (a benign race: every thread computes the same values)
    static int c_dev = -1, c_per_sm = 0, c_sms = 0;
    static size_t c_smem = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    if (dev == c_dev && smem == c_smem) {
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
        c_smem = smem;
        c_dev = dev;
    }
    const unsigned ntiles = (unsigned)(a.ny / R) * (unsigned)a.nz;
    unsigned grid = (unsigned)(per_sm * sms);
    if (grid > ntiles) grid = ntiles;
    kern<<<grid, threads, smem, st>>>(pair_args(a), make_fastdiv((unsigned)(a.ny / R)), ntiles, R, nsi);
    return cudaGetLastError();
}

// Tiles of up to 256 cells (4 consumer warps) for rows of at most 256 cells, of 384 (6 consumer
// warps, two blocks per SM) for rows of at most 384, else of 512 (8 consumer warps).
template <typename S, bool ODD, int BC, bool FORCE, int MODE>
cudaError_t step_go_stage(const StepArgs<float>& a, int nsi, cudaStream_t st)
{
    if ((a.nx * sizeof(S)) % 16 != 0 || a.nx > 512 || a.nx < 2 || nsi < 2 || nsi > 6) return cudaErrorInvalidValue;
    if (a.nx <= 256) return step_go_stage_ncw<S, ODD, BC, FORCE, MODE, 4>(a, nsi, st);
    if (a.nx <= 384) return step_go_stage_ncw<S, ODD, BC, FORCE, MODE, 6>(a, nsi, st);
    return step_go_stage_ncw<S, ODD, BC, FORCE, MODE, 8>(a, nsi, st);
}

}  // namespace fpc
