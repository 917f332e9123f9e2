// Batched complex-FP32 GEMM on the fifth-generation tensor cores (tcgen05, accumulator in
// tensor memory), with the 3xTF32 split that keeps the products near FP32 accuracy:
//     C_t = C0_t + sum_u s_u A_{t,u} Bt_{t,u}^T      (t: task, u <= 3 terms, s_u = +-1)
// A (M x K) and Bt (N x K) are row-major complex matrices (interleaved re, im); C and C0 are
// row-major or column-major.  This is the dense contraction of the block-cyclic-reduction
// factor and solve (block products of the line blocks; all right-hand sides of a system as
// the N dimension of the solve's products).
//
// Complex products as real ones: with A taken as the real M x 2K matrix of its interleaved
// entries, and each complex row b of Bt expanded into the two real rows
//     (Re b0, -Im b0, Re b1, -Im b1, ...)  and  (Im b0, Re b0, Im b1, Re b1, ...),
// the real product A_r Bt_r^T is the interleaved complex C (column 2n = Re, 2n + 1 = Im).
// Each real operand x is split into hi = tf32(x) and lo = x - hi, and the tile accumulates
// hi*hi + hi*lo + lo*hi in FP32 in tensor memory (the lo*lo term is below FP32 rounding).
//
// One CTA computes a 128 x NT complex tile (tcgen05 M = 128, N = 2 NT) of one task.  Sixteen
// operand warps load a K chunk of 16 complex columns (one 128-byte row per matrix row) from
// global memory two chunks ahead into registers (three register sets), split it and store it
// into shared memory in the 128-byte-swizzled K-major layout the tensor core reads; each warp
// then arrives on the stage's full barrier on its own (sixteen arrivals complete it).  A
// separate warp waits for it, issues the chunk's 12 MMAs from one thread and commits them to
// the stage's empty barrier, which the operand warps wait for before they overwrite the stage
// STAGES chunks later.  No CTA-wide barrier sits in the K loop.  The epilogue reads the
// accumulator with tcgen05.ld into a padded tile in the (then idle) shared memory, from which
// each warp writes whole rows (row-major C) or whole columns (column-major C), adding C0.
#include <cuda.h>   // CUtensorMap and its enums (the encoder is taken from the driver at run time)
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"
#include "trace.h"

namespace helm {

namespace {

constexpr int ZG_PRODUCERS = 512;                 // threads of the 16 operand warps
constexpr int ZG_BM = 128;   // tile rows (tcgen05 M)
constexpr int ZG_KC = 16;    // complex K per chunk: 32 floats = one 128-byte swizzle row

__device__ __forceinline__ long long zop_off(int idx, int div, long long stride, long long stride_hi) {
    return div > 0 ? (long long)(idx / div) * stride_hi + (long long)(idx % div) * stride : (long long)idx * stride;
}

constexpr int ZG_SMEM_MAX = 232448;   // dynamic + static shared memory of one CTA (227 KB)

// RING (tiles of N <= 64): a copy warp streams the raw rows of A and Bt (128 bytes of a row per
// chunk) into a ring of SLOTS shared-memory slots with bulk copies, which complete on the slot's
// mbarrier; the operand warps split from there.  Their proxy fence then orders their own stores
// only: with register-held loads it also waits for every global load the warp has in flight,
// which limits the loads to about one chunk ahead whatever the number of register sets.
template <int NT, bool RING> struct ZCfg {
    static constexpr int NR = 2 * NT;                        // real columns of the tile (tcgen05 N)
    static constexpr int A_BYTES = ZG_BM * 128;              // one split of the A chunk
    static constexpr int B_BYTES = NR * 128;                 // one split of the expanded Bt chunk
    static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int STAGES = RING ? 2 : (NT <= 64 ? 3 : 2);
    static constexpr int TMEM_COLS = NR < 32 ? 32 : NR;      // a power of two >= 32
    static constexpr int A_V4 = ZG_BM * 8 / ZG_PRODUCERS;    // float4 of the A chunk per thread
    static constexpr int B_V4 = (NT * 8 + ZG_PRODUCERS - 1) / ZG_PRODUCERS;
    static constexpr int RAW_A = ZG_BM * 128;                // raw slot: A rows, then Bt rows
    static constexpr int RAW = (ZG_BM + NT) * 128;
    static constexpr int SLOTS_FIT = (ZG_SMEM_MAX - STAGES * STAGE - 2048) / RAW;
    static constexpr int SLOTS = RING ? (SLOTS_FIT < 6 ? SLOTS_FIT : 6) : 1;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE + (RING ? (size_t)SLOTS * RAW : 0) + 1024;   // + alignment slack
    static constexpr int PW0 = RING ? 2 : 1;                 // first operand warp
    static constexpr int THREADS = ZG_PRODUCERS + 32 * PW0;  // MMA warp [, copy warp], operand warps
    // register sets of fetched chunks (register path): chunk c + NSETS - 1 is loaded while chunk
    // c is stored
    static constexpr int NSETS = 3;
};

// Tensor maps of the operands of a RING launch: each family of R x K complex matrices as a
// rank-4 float tensor (2K floats of a row, then rows, matrices of a group and groups, ordered by
// increasing stride); pos[u][role] is the dimension (1..3) of the row, in-group and group index.
struct ZMaps {
    CUtensorMap a[3], b[3];
    int8_t apos[3][3], bpos[3][3];
};

// tiled tensor copy of one box into this CTA's shared memory, completing its bytes on the mbarrier
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float4 ld_shared_v4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr)
                 : "memory");
    return v;
}

template <int NT, bool RING>
__global__ void __launch_bounds__(ZCfg<NT, RING>::THREADS, 1)
    zgemm_tc_kernel(ZGemmArgs a, const __grid_constant__ ZMaps maps) {
    using Cfg = ZCfg<NT, RING>;
    static_assert(!RING || Cfg::SLOTS >= 2, "the ring needs two slots");
    extern __shared__ uint8_t zg_smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[Cfg::STAGES];    // stage written (one arrival per operand warp)
    __shared__ __align__(8) uint64_t empty_bar[Cfg::STAGES];   // stage read by its MMAs (commit)
    __shared__ __align__(8) uint64_t raw_full[Cfg::SLOTS];     // ring slot's copies landed (RING)
    __shared__ __align__(8) uint64_t raw_empty[Cfg::SLOTS];    // ring slot read by every operand warp (RING)
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    if (a.skip && *a.skip) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * ZG_BM, n0 = blockIdx.y * NT;
    const int ks = a.ksplit, kpart = (int)(blockIdx.z % (unsigned)ks);   // split-K part of this CTA
    const int* task = a.tasks + (size_t)(blockIdx.z / (unsigned)ks) * 8;
    if (a.sys_frozen && a.sys_frozen[2 * (task[7] / a.sys_div)]) return;   // its system needs no correction
    const uint32_t smem0 = (smem_u32(zg_smem_raw) + 1023u) & ~1023u;
    const uint32_t ring0 = smem0 + (uint32_t)(Cfg::STAGES * Cfg::STAGE);   // raw slots (RING)

    // active terms (a term whose A index is negative is absent)
    int act[3] = {0, 0, 0}, nterms = 0;
    for (int u = 0; u < a.nterms; ++u)
        if (task[u] >= 0) act[nterms++] = u;
    const int nkc = (a.K + ZG_KC - 1) / ZG_KC;
    // this CTA's K chunks [cbase, cbase + nchunks) of the task's nterms * nkc (all of them
    // unless split); the loops below count chunks locally from 0
    const int cbase = (int)((long long)kpart * nterms * nkc / ks);
    const int nchunks = (int)((long long)(kpart + 1) * nterms * nkc / ks) - cbase;

    const bool mma_warp = warp == 0;
    const int ptid = tid - 32 * Cfg::PW0;   // operand-thread index (warps PW0 .. PW0 + 15)
    if (tid == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            mbar_init(&full_bar[s], ZG_PRODUCERS / 32);   // one arrival per operand warp
            mbar_init(&empty_bar[s], 1);
        }
        if (RING)
            for (int q = 0; q < Cfg::SLOTS; ++q) {
                mbar_init(&raw_full[q], 1);                     // the copy warp's expect_tx arrival
                mbar_init(&raw_empty[q], ZG_PRODUCERS / 32);    // one arrival per operand warp
            }
        mbar_init(&done_bar, 1);
        fence_mbar_init_cluster();
        s_abort = 0;
    }
    if (mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"((uint32_t)Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // ---- operand fetch of one chunk into registers (chunk c + NSETS - 1 is fetched while chunk c
    // is stored, so that a load has NSETS - 1 chunks of work to arrive in)
    using RA = float4[Cfg::A_V4];
    using RB = float4[Cfg::B_V4];
    auto term_of = [&](int c) { const int cu = c / nkc; return cu == 0 ? act[0] : (cu == 1 ? act[1] : act[2]); };
    auto fetch = [&](int c, RA &ra, RB &rb) {
        const int u = term_of(cbase + c), k0 = ((cbase + c) % nkc) * ZG_KC;
        const float2 *A = a.A[u].base + zop_off(task[u], a.A[u].div, a.A[u].stride, a.A[u].stride_hi);
        const float2 *B = a.B[u].base + zop_off(task[3 + u], a.B[u].div, a.B[u].stride, a.B[u].stride_hi);
#pragma unroll
        for (int i = 0; i < Cfg::A_V4; ++i) {
            const int e = ptid + i * ZG_PRODUCERS, r = e >> 3, k = k0 + 2 * (e & 7);
            ra[i] = (m0 + r < a.M && k < a.K)
                        ? __ldg(reinterpret_cast<const float4 *>(A + (long long)(m0 + r) * a.A[u].ld + k))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < Cfg::B_V4; ++i) {
            const int e = ptid + i * ZG_PRODUCERS, n = e >> 3, k = k0 + 2 * (e & 7);
            rb[i] = (e < NT * 8 && n0 + n < a.N && k < a.K)
                        ? __ldg(reinterpret_cast<const float4 *>(B + (long long)(n0 + n) * a.B[u].ld + k))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    // ---- split and store of a fetched chunk into stage s
    auto store = [&](int c, int s, const RA &ra, const RB &rb) {
        const float sg = a.sign[term_of(cbase + c)];
        const uint32_t base = smem0 + (uint32_t)(s * Cfg::STAGE);
        const uint32_t a_hi = base, a_lo = base + Cfg::A_BYTES;
        const uint32_t b_hi = base + 2 * Cfg::A_BYTES, b_lo = b_hi + Cfg::B_BYTES;
#pragma unroll
        for (int i = 0; i < Cfg::A_V4; ++i) {
            const int e = ptid + i * ZG_PRODUCERS, r = e >> 3, j = e & 7;
            float4 hi, lo;
            split4(ra[i], sg, hi, lo);
            st_shared_v4(a_hi + sw128(r, j), hi);
            st_shared_v4(a_lo + sw128(r, j), lo);
        }
#pragma unroll
        for (int i = 0; i < Cfg::B_V4; ++i) {
            const int e = ptid + i * ZG_PRODUCERS, n = e >> 3, j = e & 7;
            if (e < NT * 8) {
                const float4 v = rb[i];
                float4 hi, lo;
                // real row 2n: (Re, -Im) pairs; real row 2n + 1: (Im, Re) pairs
                split4(make_float4(v.x, -v.y, v.z, -v.w), 1.f, hi, lo);
                st_shared_v4(b_hi + sw128(2 * n, j), hi);
                st_shared_v4(b_lo + sw128(2 * n, j), lo);
                split4(make_float4(v.y, v.x, v.w, v.z), 1.f, hi, lo);
                st_shared_v4(b_hi + sw128(2 * n + 1, j), hi);
                st_shared_v4(b_lo + sw128(2 * n + 1, j), lo);
            }
        }
    };

    // ---- RING: the chunk from its raw slot (rows of 128 bytes as copied) into registers
    auto fetch_raw = [&](int c, RA &ra, RB &rb) {
        const int k0 = ((cbase + c) % nkc) * ZG_KC;
        const uint32_t slot = ring0 + (uint32_t)((c % Cfg::SLOTS) * Cfg::RAW);
#pragma unroll
        for (int i = 0; i < Cfg::A_V4; ++i) {
            const int e = ptid + i * ZG_PRODUCERS, r = e >> 3, j = e & 7;
            ra[i] = (m0 + r < a.M && k0 + 2 * j < a.K) ? ld_shared_v4(slot + (uint32_t)(r * 128 + j * 16))
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < Cfg::B_V4; ++i) {
            const int e = ptid + i * ZG_PRODUCERS, n = e >> 3, j = e & 7;
            rb[i] = (e < NT * 8 && n0 + n < a.N && k0 + 2 * j < a.K)
                        ? ld_shared_v4(slot + (uint32_t)(Cfg::RAW_A + n * 128 + j * 16))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };

    constexpr uint32_t idesc = idesc_tf32(Cfg::NR);
    auto give_up = [&]() {
        atomicOr(a.status, ST_TIMEOUT);
        s_abort = 1;
    };
    if (warp >= Cfg::PW0 && !RING) {
        // operand warps: chunk c waits for its stage to be free, is split and stored, chunk c + 2
        // is fetched into the freed registers, and every warp arrives on the stage's full barrier
        // (16 arrivals complete it) without waiting for the other warps; they run up to STAGES
        // chunks ahead of the tensor core.  Decisions to stop are taken per warp (votes), so that
        // no lane leaves the loop while its warp's other lanes go on
        auto pstep = [&](int c, RA &ra, RB &rb, RA &na, RB &nb) -> bool {
            const int s = c % Cfg::STAGES;
            const bool bad = c >= Cfg::STAGES &&
                             !mbar_wait_or_abort(&empty_bar[s], (uint32_t)((c / Cfg::STAGES - 1) & 1), a.tries, &s_abort);
            if (__any_sync(0xffffffffu, bad)) {   // a warp whose wait gave up writes no stage the MMAs may read
                if (bad) give_up();
                return false;
            }
            store(c, s, ra, rb);
            // the stores are made visible to the tensor core's (async proxy) reads before the
            // next loads are issued: a proxy fence after them would wait for those loads as well
            // and expose their latency on every chunk
            fence_proxy_async_smem();
            if (c + Cfg::NSETS - 1 < nchunks) fetch(c + Cfg::NSETS - 1, na, nb);
            __syncwarp();   // every lane's stores and fence before the warp's arrival
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[s])) : "memory");
            return !__any_sync(0xffffffffu, *(volatile int *)&s_abort);
        };
        // NSETS register sets: chunk c is stored from set c mod NSETS while chunk c + NSETS - 1 is
        // loaded into set (c - 1) mod NSETS, whose stores (chunk c - 1) have been issued -- loading
        // into the set being stored would wait for the stores to read their registers
        constexpr int NS = Cfg::NSETS;
        float4 ra[NS][Cfg::A_V4], rb[NS][Cfg::B_V4];
#pragma unroll
        for (int i = 0; i < NS - 1; ++i)
            if (i < nchunks) fetch(i, ra[i], rb[i]);
        bool go = true;
        for (int c0 = 0; go && c0 < nchunks; c0 += NS) {
#pragma unroll
            for (int i = 0; i < NS; ++i)
                if (go && c0 + i < nchunks) go = pstep(c0 + i, ra[i], rb[i], ra[(i + NS - 1) % NS], rb[(i + NS - 1) % NS]);
        }
    } else if (warp >= Cfg::PW0) {
        // RING operand warps: chunk c waits for its raw slot and its stage, is split from the
        // slot into the stage, and the warp arrives on the stage's full barrier and on the slot's
        // empty barrier (16 arrivals each), without waiting for the other warps
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % Cfg::STAGES, q = c % Cfg::SLOTS;
            bool bad = !mbar_wait_or_abort(&raw_full[q], (uint32_t)((c / Cfg::SLOTS) & 1), a.tries, &s_abort);
            if (!bad && c >= Cfg::STAGES)
                bad = !mbar_wait_or_abort(&empty_bar[s], (uint32_t)((c / Cfg::STAGES - 1) & 1), a.tries, &s_abort);
            if (__any_sync(0xffffffffu, bad)) {
                if (bad) give_up();
                break;
            }
            float4 ra[Cfg::A_V4], rb[Cfg::B_V4];
            fetch_raw(c, ra, rb);
            store(c, s, ra, rb);
            fence_proxy_async_smem();   // the stores, before the tensor core reads them
            __syncwarp();               // every lane's slot reads, stores and fence before the arrivals
            if (lane == 0) {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[s])) : "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&raw_empty[q])) : "memory");
            }
            if (__any_sync(0xffffffffu, *(volatile int *)&s_abort)) break;
        }
    } else if (RING && warp == 1) {
        // RING copy warp: chunk c (a box of 128 rows of A and one of NT rows of Bt, 32 floats of K
        // each, rows and K beyond the matrices filled with zeros) into slot c mod SLOTS once every
        // operand warp has read the slot's previous chunk; the slot's mbarrier completes when both
        // boxes have landed
        int issued = 0;
        for (int c = 0; c < nchunks; ++c) {
            const int q = c % Cfg::SLOTS;
            if (__any_sync(0xffffffffu, *(volatile int *)&s_abort)) break;
            if (c >= Cfg::SLOTS) {
                const bool ok = mbar_wait_or_abort(&raw_empty[q], (uint32_t)((c / Cfg::SLOTS - 1) & 1), a.tries, &s_abort);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) give_up();
                    break;
                }
            }
            if (lane == 0) {
                const int u = term_of(cbase + c), k0 = ((cbase + c) % nkc) * ZG_KC;
                const uint32_t slot = ring0 + (uint32_t)(q * Cfg::RAW);
                mbar_arrive_expect_tx(&raw_full[q], (uint32_t)Cfg::RAW);
                int ca[4] = {2 * k0, 0, 0, 0}, cb[4] = {2 * k0, 0, 0, 0};
                const int ia = task[u], ib = task[3 + u];
                ca[maps.apos[u][0]] = m0;
                ca[maps.apos[u][1]] = a.A[u].div > 0 ? ia % a.A[u].div : ia;
                ca[maps.apos[u][2]] = a.A[u].div > 0 ? ia / a.A[u].div : 0;
                cb[maps.bpos[u][0]] = n0;
                cb[maps.bpos[u][1]] = a.B[u].div > 0 ? ib % a.B[u].div : ib;
                cb[maps.bpos[u][2]] = a.B[u].div > 0 ? ib / a.B[u].div : 0;
                tma_load_4d(slot, &maps.a[u], ca[0], ca[1], ca[2], ca[3], &raw_full[q]);
                tma_load_4d(slot + Cfg::RAW_A, &maps.b[u], cb[0], cb[1], cb[2], cb[3], &raw_full[q]);
            }
            __syncwarp();
            issued = c + 1;
        }
        // no copy may land in shared memory after the CTA has left: the last ones (one per slot)
        // are waited for, also after an abort
        for (int c = issued > Cfg::SLOTS ? issued - Cfg::SLOTS : 0; c < issued; ++c)
            mbar_wait_bounded(&raw_full[c % Cfg::SLOTS], (uint32_t)((c / Cfg::SLOTS) & 1), a.tries);
    } else if (warp == 0 && lane == 0) {
        // MMA thread: 12 MMAs per chunk (3 split products x 4 K steps), committed to the stage's
        // empty barrier; then one commit that covers every MMA issued
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % Cfg::STAGES;
            if (!mbar_wait_or_abort(&full_bar[s], (uint32_t)((c / Cfg::STAGES) & 1), a.tries, &s_abort)) {
                give_up();
                break;
            }
            tc_fence_after();
            const uint32_t base = smem0 + (uint32_t)(s * Cfg::STAGE);
            const uint32_t a_hi = base, a_lo = base + Cfg::A_BYTES;
            const uint32_t b_hi = base + 2 * Cfg::A_BYTES, b_lo = b_hi + Cfg::B_BYTES;
#pragma unroll
            for (int p = 0; p < 3; ++p) {   // hi*hi, hi*lo, lo*hi
                const uint32_t aa = p == 2 ? a_lo : a_hi, bb = p == 1 ? b_lo : b_hi;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)   // K = 8 TF32 (32 bytes) per instruction
                    tc_mma(tmem, desc_sw128(aa + 32 * kk), desc_sw128(bb + 32 * kk), idesc,
                           (c > 0 || p > 0 || kk > 0) ? 1u : 0u);
            }
            tc_commit(&empty_bar[s]);
        }
        tc_commit(&done_bar);
    }
    // every MMA issued is complete before the accumulator is read or freed
    if (!mbar_wait_bounded(&done_bar, 0, a.tries)) give_up();
    tc_fence_after();
    const bool aborted = __syncthreads_or(*(volatile int *)&s_abort);
    const bool ok = !aborted && nchunks > 0;
    // a split part without chunks still owes its (zero) partial tile
    const bool zero_part = !aborted && nchunks == 0 && ks > 1;

    if ((ok || zero_part) && warp >= Cfg::PW0) {
        // Epilogue through shared memory (free once every MMA is complete): the operand warps
        // copy the accumulator tile from tensor memory (warp w: lanes 32 (w % 4) .. + 31, the
        // real columns of part (w - 1) / 4) into a padded [128][NT + 1] complex tile, meet, and
        // write C (adding C0) a row or a column per warp and step, so that every warp store
        // covers consecutive addresses whether C is row- or column-major.
        constexpr int parts = Cfg::NR >= 64 ? 4 : Cfg::NR / 16, cpp = Cfg::NR / parts, TS = NT + 1;
        float2 *T = reinterpret_cast<float2 *>(zg_smem_raw + (smem0 - smem_u32(zg_smem_raw)));
        const int q = warp & 3, pw = warp - Cfg::PW0, h = pw >> 2;
        if (h < parts) {
            const int r = 32 * q + lane;
            for (int col = h * cpp; col < (h + 1) * cpp; col += 16) {
                float v[16];
                if (ok) {
                    tc_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col, v);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = 0.f;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) T[r * TS + col / 2 + i] = make_float2(v[2 * i], v[2 * i + 1]);
            }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(ZG_PRODUCERS) : "memory");
        // split parts write their partial tile (C's layout, leading dimension M or N, no C0)
        const bool split = ks > 1;
        const float2 *C0 = (!split && a.C0.base)
                               ? a.C0.base + zop_off(task[6], a.C0.div, a.C0.stride, a.C0.stride_hi)
                               : nullptr;
        float2 *C = split ? a.part + (size_t)blockIdx.z * ((size_t)a.M * a.N)
                          : a.C + zop_off(task[7], a.c_div, a.c_stride, a.c_stride_hi);
        const long long ldc = split ? (a.c_col ? a.M : a.N) : a.ldc;
        if (!a.c_col) {
            for (int rr = pw; rr < ZG_BM; rr += ZG_PRODUCERS / 32) {   // row-major: a row per warp
                const int m = m0 + rr;
                if (m >= a.M) break;
                for (int nn = lane; nn < NT && n0 + nn < a.N; nn += 32) {
                    float2 out = T[rr * TS + nn];
                    if (C0) {
                        const float2 b = C0[(long long)m * a.C0.ld + n0 + nn];
                        out.x += b.x;
                        out.y += b.y;
                    }
                    C[(long long)m * ldc + n0 + nn] = out;
                }
            }
        } else {
            for (int nn = pw; nn < NT; nn += ZG_PRODUCERS / 32) {     // column-major: a column per warp
                const int n = n0 + nn;
                if (n >= a.N) break;
                for (int rr = lane; rr < ZG_BM && m0 + rr < a.M; rr += 32) {
                    float2 out = T[rr * TS + nn];
                    if (C0) {
                        const float2 b = C0[(long long)n * a.C0.ld + m0 + rr];
                        out.x += b.x;
                        out.y += b.y;
                    }
                    C[(long long)n * ldc + m0 + rr] = out;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (mma_warp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)Cfg::TMEM_COLS)
                     : "memory");
}

// C_t = C0_t + sum over the ksplit partial tiles of task t, in part order; one thread per element
// of C, consecutive threads along C's contiguous dimension
__global__ void zsplit_reduce_kernel(ZGemmArgs a) {
    if (a.skip && *a.skip) return;   // the GEMM itself was skipped
    const int *task = a.tasks + (size_t)blockIdx.y * 8;
    if (a.sys_frozen && a.sys_frozen[2 * (task[7] / a.sys_div)]) return;
    const long long mn = (long long)a.M * a.N;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mn) return;
    const int inner = a.c_col ? a.M : a.N;   // C's contiguous dimension
    const int i = (int)(e / inner), o = (int)(e % inner);
    const float2 *P = a.part + (size_t)blockIdx.y * a.ksplit * mn + e;
    float2 v = P[0];
    for (int p = 1; p < a.ksplit; ++p) {
        const float2 w = P[(size_t)p * mn];
        v.x += w.x;
        v.y += w.y;
    }
    if (a.C0.base && task[6] >= 0) {
        const float2 b = a.C0.base[zop_off(task[6], a.C0.div, a.C0.stride, a.C0.stride_hi) + (long long)i * a.C0.ld + o];
        v.x += b.x;
        v.y += b.y;
    }
    a.C[zop_off(task[7], a.c_div, a.c_stride, a.c_stride_hi) + (long long)i * a.ldc + o] = v;
}

// streaming multiprocessors of the current device (queried once)
int num_sms() {
    static const int n = []() {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            v = 0;
        cudaGetLastError();
        return v > 0 ? v : 148;
    }();
    return n;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder (looked up once; null if the driver does not provide it)
EncodeTiledFn tensor_map_encoder() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Tensor map of a family of R x K complex matrices (see ZMaps) with boxes of 32 floats x
// box_rows rows; false if the family cannot be described (unknown count, strides that are not
// multiples of 16 bytes) or the encoder refuses it.
bool encode_family(CUtensorMap *m, int8_t pos[3], const ZOperand &o, int R, int K, int box_rows) {
    const EncodeTiledFn enc = tensor_map_encoder();
    if (!enc || !o.base || o.count <= 0 || o.ld < K) return false;
    struct Dim { unsigned long long ext, stride; int role; };
    Dim d[3];
    d[0] = {(unsigned long long)R, (unsigned long long)o.ld * 8ull, 0};
    if (o.div > 0) {
        d[1] = {(unsigned long long)o.div, (unsigned long long)o.stride * 8ull, 1};
        d[2] = {(unsigned long long)o.count, (unsigned long long)o.stride_hi * 8ull, 2};
    } else {
        d[1] = {(unsigned long long)o.count, (unsigned long long)o.stride * 8ull, 1};
        d[2] = {1ull, 0ull, 2};
    }
    // dimensions of one element last, the others by increasing stride; a dimension of one
    // element takes the stride that nests it after the previous one
    std::stable_sort(d, d + 3, [](const Dim &x, const Dim &y) {
        if ((x.ext == 1) != (y.ext == 1)) return y.ext == 1;
        return x.stride < y.stride;
    });
    cuuint64_t dims[4] = {(cuuint64_t)2 * K, 0, 0, 0}, strides[3];
    cuuint32_t box[4] = {32, 1, 1, 1}, estr[4] = {1, 1, 1, 1};
    unsigned long long prev = (unsigned long long)2 * K * 4, prev_ext = 1;
    for (int i = 0; i < 3; ++i) {
        unsigned long long st = d[i].ext == 1 ? prev * prev_ext : d[i].stride;
        if (st == 0 || (st & 15) || st >= (1ull << 40) || d[i].ext > (1ull << 32)) return false;
        dims[i + 1] = d[i].ext;
        strides[i] = st;
        if (d[i].role == 0) box[i + 1] = (cuuint32_t)box_rows;
        pos[d[i].role] = (int8_t)(i + 1);
        prev = st;
        prev_ext = d[i].ext;
    }
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2 *>(o.base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT, bool RING> cudaError_t launch_nt(const ZGemmArgs &a, const ZMaps &maps, int n_tasks, cudaStream_t st) {
    using Cfg = ZCfg<NT, RING>;
    const void *fn = (const void *)zgemm_tc_kernel<NT, RING>;
    cudaError_t e = ensure_dyn_smem(fn, Cfg::SMEM);
    if (e != cudaSuccess) return e;
    // split-K where the launch fills at most half of the SMs: as many parts as keep it within one
    // wave, at most one part per K chunk of a term, within the partial buffer
    ZGemmArgs b = a;
    b.ksplit = 1;
    const long long tiles = (long long)((a.M + ZG_BM - 1) / ZG_BM) * ((a.N + NT - 1) / NT) * n_tasks;
    const int kNumSMs = num_sms();
    if (a.part && tiles * 2 <= kNumSMs) {
        const int nkc = (a.K + ZG_KC - 1) / ZG_KC;
        long long ks = std::min<long long>(nkc, kNumSMs / tiles);
        ks = std::min<long long>(ks, (long long)(a.part_cap / ((size_t)a.M * a.N * n_tasks)));
        ks = std::min<long long>(ks, 65535 / n_tasks);
        if (ks >= 2) b.ksplit = (int)ks;
    }
    dim3 grid((unsigned)((a.M + ZG_BM - 1) / ZG_BM), (unsigned)((a.N + NT - 1) / NT), (unsigned)(n_tasks * b.ksplit));
    HELM_TRACED_W(K_ZGEMM, st, a.flops, (zgemm_tc_kernel<NT, RING><<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(b, maps)));
    if (b.ksplit > 1) {
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const long long mn = (long long)a.M * a.N;
        dim3 rg((unsigned)((mn + 255) / 256), (unsigned)n_tasks);
        HELM_TRACED(K_ZSPLIT, st, (zsplit_reduce_kernel<<<rg, 256, 0, st>>>(b)));
    }
    return cudaGetLastError();
}

// narrow tiles: the tensor-copy ring when every operand family has a tensor map, else the
// register path
template <int NT> cudaError_t launch_narrow(const ZGemmArgs &a, int n_tasks, cudaStream_t st) {
    ZMaps maps{};
    bool ring = true;
    for (int u = 0; ring && u < a.nterms; ++u)
        ring = encode_family(&maps.a[u], maps.apos[u], a.A[u], a.M, a.K, ZG_BM) &&
               encode_family(&maps.b[u], maps.bpos[u], a.B[u], a.N, a.K, NT);
    return ring ? launch_nt<NT, true>(a, maps, n_tasks, st) : launch_nt<NT, false>(a, maps, n_tasks, st);
}

}  // namespace

cudaError_t launch_zgemm(const ZGemmArgs &a, int n_tasks, cudaStream_t st) {
    if (n_tasks <= 0) return cudaSuccess;
    if (a.M <= 0 || a.N <= 0 || a.K <= 0 || (a.K & 1) || a.nterms < 1 || a.nterms > 3 || n_tasks > 65535)
        return cudaErrorInvalidValue;
    for (int u = 0; u < a.nterms; ++u)   // 16-byte operand loads: even leading dimensions and offsets
        if ((a.A[u].ld & 1) || (a.B[u].ld & 1) || (a.A[u].stride & 1) || (a.B[u].stride & 1) ||
            (a.A[u].stride_hi & 1) || (a.B[u].stride_hi & 1) || ((uintptr_t)a.A[u].base & 15) ||
            ((uintptr_t)a.B[u].base & 15))
            return cudaErrorInvalidValue;
    if (a.N <= 16) return launch_narrow<16>(a, n_tasks, st);
    if (a.N <= 32) return launch_narrow<32>(a, n_tasks, st);
    if (a.N <= 64) return launch_narrow<64>(a, n_tasks, st);
    return launch_nt<128, false>(a, ZMaps{}, n_tasks, st);
}

}  // namespace helm
