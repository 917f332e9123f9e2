// Shared device helpers for libhelm: complex arithmetic on interleaved pairs, the
// grid coefficients of the discrete operator, and thread-block-cluster primitives.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace helm {

// ------------------------------------------------------------------ complex types
template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
template <typename T> using cx_t = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ cx_t<T> mkc(T re, T im) {
    cx_t<T> z; z.x = re; z.y = im; return z;
}
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
    V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename V> __host__ __device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
// acc += a * b
template <typename V> __host__ __device__ __forceinline__ void cfma(V &acc, V a, V b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
template <typename V> __host__ __device__ __forceinline__ void cfms(V &acc, V a, V b) {
    acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }

__device__ __forceinline__ float2 to_c64(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_c128(float2 a) { return make_double2((double)a.x, (double)a.y); }

template <typename V> __device__ __forceinline__ V ldcg(const V *p);
template <> __device__ __forceinline__ double2 ldcg<double2>(const double2 *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float2 ldcg<float2>(const float2 *p) { return __ldcg(p); }

// ----------------------------------------------------------- grid coefficients
// Uniform grid, node (i, j) at (i hx, j hz), k = i*nz + j.  Edge couplings of the
// five-point P1 stiffness: horizontal (i-1,j)-(i,j) is -(hz/hx) w_z(j), vertical
// (i,j)-(i,j+1) is -(hx/hz) w_x(i), where the weight is 1/2 for an edge lying on the
// boundary and 1 otherwise.
struct GridGeom {
    int nx, nz;
    double hx, hz;
    int lump = 0;   // mass lumping: 0 tensor trapezoid, 1 / 2 triangles cut (i,j)-(i+1,j+1) / (i+1,j)-(i,j+1)
};

__host__ __device__ __forceinline__ double edge_w(int idx, int n) { return (idx == 0 || idx == n - 1) ? 0.5 : 1.0; }

// lumped mass d_k of node (i, j) (Appendix "Numerical forward model", nodal quadrature): the tensor
// trapezoid hx hz q(i) q(j), or the vertex quadrature of the triangles (a third of each adjacent
// triangle's area), which differs from it only at the four grid corners: hx hz / 3 where the cutting
// diagonal ends, hx hz / 6 at the other two
__host__ __device__ __forceinline__ double lumped_mass(const GridGeom &g, int i, int j) {
    const bool ci = i == 0 || i == g.nx - 1, cj = j == 0 || j == g.nz - 1;
    if (g.lump == 0 || !(ci && cj)) return g.hx * g.hz * edge_w(i, g.nx) * edge_w(j, g.nz);
    const bool diag_end = (i == 0) == (j == 0);   // (0,0) or (nx-1,nz-1): ends of the "up" diagonal
    return g.hx * g.hz / ((diag_end == (g.lump == 1)) ? 3.0 : 6.0);
}

// coupling between line i-1 and line i at row j (i >= 1)
__host__ __device__ __forceinline__ double coup_x(const GridGeom &g, int j) { return -(g.hz / g.hx) * edge_w(j, g.nz); }
// coupling between rows j and j+1 of line i (j <= nz-2)
__host__ __device__ __forceinline__ double coup_z(const GridGeom &g, int i) { return -(g.hx / g.hz) * edge_w(i, g.nx); }

// ------------------------------------------------------------ cluster primitives
__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r; asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r)); return r;
}
__device__ __forceinline__ unsigned cluster_id_x() {
    unsigned r; asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r)); return r;
}
// Hardware cluster barrier with release/acquire ordering at cluster scope: global
// stores made by any thread of the cluster before the barrier are visible to loads
// of every thread of the cluster after it.  All threads of all CTAs must reach it.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// device status bits (OR-ed together)
enum : int { ST_SINGULAR = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4 };

}  // namespace helm

namespace helm {
// ------------------------------------------------- shared-memory / async-copy helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// address of the same shared-memory offset in CTA `rank` of this cluster
__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, double2 v) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(v.x), "d"(v.y) : "memory");
}
// split cluster barrier: arrive (release) and wait (acquire)
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

// asynchronous global -> shared copies of one complex element (8 or 16 bytes)
__device__ __forceinline__ void cp_async_elem(float2 *dst, const float2 *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2 *dst, const double2 *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
}  // namespace helm

namespace helm {
// ------------------------------------------------------------------ mbarriers
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init_cluster() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// arrive (release, cluster scope) on an mbarrier of another CTA of the cluster (mapa address)
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on the phase with the given parity; false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t max_tries) {
    for (uint32_t t = 0; t < max_tries; ++t)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// bounded wait that also gives up as soon as the CTA's abort word is set (by this CTA or,
// remotely, by another CTA of the cluster that gave up first)
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, uint32_t max_tries,
                                                   const int *abort_word) {
    for (uint32_t t = 0; t < max_tries; ++t) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*(const volatile int *)abort_word) return false;
    }
    return false;
}
// Abort protocol of the cluster kernels.  A CTA whose bounded wait gives up sets the abort word
// (a __shared__ int at the same offset in every CTA) in every CTA of its cluster, so that the
// others stop waiting and stop producing.  No CTA leaves before the final cluster barrier,
// which every CTA reaches in bounded time since every wait is bounded; after it a CTA whose
// abort word is set waits a fixed drain time, so that asynchronous stores and bulk copies that
// peers issued before they saw the word land in (or finish reading) shared memory that is still
// alive.
__device__ __forceinline__ void cluster_abort_broadcast(int *abort_word, unsigned cluster_ctas) {
    const uint32_t a = smem_u32(abort_word);
    for (unsigned r = 0; r < cluster_ctas; ++r)
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(mapa_u32(a, r)), "r"(1) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr uint64_t kAbortDrainNs = 50000;   // 50 us: far beyond the latency of an in-flight copy
__device__ __forceinline__ void abort_drain() {
    const uint64_t t0 = global_ns();
    while (global_ns() - t0 < kAbortDrainNs) __nanosleep(1000);
}
// default try count of the bounded mbarrier waits (each try suspends for a hardware time
// limit, so this is seconds at worst); helm_set_wait_tries overrides it for later launches
constexpr uint32_t kDefaultWaitTries = 1u << 22;
uint32_t wait_tries();   // host: the try count the next launches take
uint32_t fault_flags();  // host: HELM_FAULT_* bits of the HELM_FAULT environment variable
// asynchronous store into another CTA's shared memory that completes `bytes` of the
// transaction count of the mbarrier at remote shared address `rbar`
__device__ __forceinline__ void st_async(uint32_t raddr, float2 v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "f"(v.x), "f"(v.y), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void st_async(uint32_t raddr, double2 v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "d"(v.x), "d"(v.y), "r"(rbar)
                 : "memory");
}
}  // namespace helm

namespace helm {
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
}  // namespace helm

namespace helm {
// bulk copy (TMA engine) of `bytes` from this CTA's shared memory to another CTA's shared
// memory (raddr, from mapa), completing `bytes` of the transaction count of the mbarrier at
// remote address rbar.  bytes: multiple of 16; both addresses 16-byte aligned.
__device__ __forceinline__ void bulk_copy_s2s(uint32_t raddr, uint32_t laddr, uint32_t bytes, uint32_t rbar) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(raddr), "r"(laddr), "r"(bytes), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
}  // namespace helm
