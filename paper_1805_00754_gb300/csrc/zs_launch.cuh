// zs_launch.cuh - host-side launch helpers shared by the launcher translation
// units (zs_compress_*.cu, zs_query_*.cu): shared-memory opt-in, the
// tensor-path scratch carving and launch sequence, and the query launch set.
#pragma once

#include <algorithm>
#include <climits>
#include <cstring>
#include <type_traits>

#include <cudaTypedefs.h>

#include "zs_kernels_dev.cuh"
#include "zs_prof.h"

namespace zs {

// Opt in to the dynamic shared memory a launch needs (static + dynamic may not
// exceed 48 KB without it).
template <typename K>
static cudaError_t set_smem(K kern, size_t bytes) {
    if (bytes <= 32 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define ZS_TRY(x)                                  \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return e_;          \
    } while (0)

// ---------------------------------------------------------------------------
// Tensor-core path (see zs_tc_kernels.cuh).
// ---------------------------------------------------------------------------
static inline size_t tc_subspace_smem(int n, int m, bool& yglob) {
    const size_t both = (size_t)2 * n * (m + 1) * 4;
    yglob = both > 110 * 1024;
    return yglob ? (size_t)n * (m + 1) * 4 : both;
}

// Auxiliary scratch of the tensor path, carved from one buffer:
// [Hp: tiles x m x m | Cq: items x m x m | Zs: items x m x kw | th: items x kw |
//  thm: items x m | list: 2 + items ints]

static inline void tc_aux_carve(void* aux, int64_t items, int64_t tiles, int m, int kw, TcScratch& sc) {
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    char* p = (char*)aux;
    sc.Hp = (float*)p;
    p += r(4 * (size_t)tiles * m * m);
    sc.Cq = (float*)p;
    p += r(4 * (size_t)items * m * m);
    sc.Zs = (float*)p;
    p += r(4 * (size_t)items * m * kw);
    sc.th = (float*)p;
    p += r(4 * (size_t)items * kw);
    sc.thm = (float*)p;
    p += r(4 * (size_t)items * m);
    sc.list = (int*)p;
    p += r(4 * (size_t)(items + 2));
    sc.cplan = (int*)p;
}

// The sketch kernel covers n <= 512 with its accumulator S (n x m) held in
// registers: 16 NMT rows per warp, m <= MB.
static inline bool sketch_fits(int n, int m, bool query = false) {
    // Storage blocks with n > 256 and m > 32 stay on the bf16-Gram route:
    // its subspace (pivoted columns and a power step) is one power of X^T X
    // ahead of the sketch's, and on the precision workload (k = 32 of 40
    // signal directions) the sketch left ~96% of the blocks to k_refine
    // (measured: 20 GB/s against 61 GB/s).  Stacked query matrices pass the
    // accuracy test from the sketch, which there beats the Gram route.
    if (n > 512 || (!query && n > 256 && m > 32)) return false;
    return sketch_smem(n, m).total <= 227 * 1024 && (size_t)n * (m + 1) * 4 <= 227 * 1024;
}

template <class Src, typename Tin, int NMT, int MB>
static cudaError_t sketch_launch(const Src& src, const TcScratch& sc, int n, int max_items, cudaStream_t st) {
    const size_t sm = sketch_smem(n, sc.m).total;
    ZS_TRY(set_smem(k_sketch<Src, Tin, NMT, MB>, sm));
    k_sketch<Src, Tin, NMT, MB><<<max_items * kSketchCL, 256, sm, st>>>(src, sc, n);
    return cudaGetLastError();
}

template <class Src, typename Tin>
static cudaError_t sketch_dispatch(const Src& src, const TcScratch& sc, int n, int max_items, cudaStream_t st) {
    if (n <= 128) return sc.m <= 32 ? sketch_launch<Src, Tin, 1, 32>(src, sc, n, max_items, st)
                                    : sketch_launch<Src, Tin, 1, 64>(src, sc, n, max_items, st);
    if (n <= 256) return sc.m <= 32 ? sketch_launch<Src, Tin, 2, 32>(src, sc, n, max_items, st)
                                    : sketch_launch<Src, Tin, 2, 64>(src, sc, n, max_items, st);
    return sc.m <= 32 ? sketch_launch<Src, Tin, 4, 32>(src, sc, n, max_items, st)
                      : sketch_launch<Src, Tin, 4, 64>(src, sc, n, max_items, st);
}

template <class Src, int RPL, int CPW>
static cudaError_t orth_launch(const Src& src, const TcScratch& sc, int n, int max_items, cudaStream_t st) {
    const size_t sm = (size_t)n * (sc.m + 1) * 4;
    ZS_TRY(set_smem(k_orth<Src, RPL, CPW>, sm));
    k_orth<Src, RPL, CPW><<<max_items, 32 * kOrthWarps, sm, st>>>(src, sc, n);
    return cudaGetLastError();
}

// rows per lane RPL = n / 32 (n <= 512), columns per warp CPW = m / 16
template <class Src>
static cudaError_t orth_dispatch(const Src& src, const TcScratch& sc, int n, int max_items, cudaStream_t st) {
    if (n <= 256) return sc.m <= 32 ? orth_launch<Src, 8, 2>(src, sc, n, max_items, st)
                                    : orth_launch<Src, 8, 4>(src, sc, n, max_items, st);
    return sc.m <= 32 ? orth_launch<Src, 16, 2>(src, sc, n, max_items, st)
                      : orth_launch<Src, 16, 4>(src, sc, n, max_items, st);
}

// cuTensorMapEncodeTiled from the driver (null where the driver has none)
static PFN_cuTensorMapEncodeTiled_v12000 t5_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}
// rows x n fp32 matrix (row stride ld elements) read in 32 x box_rows boxes, 128-byte swizzle
static bool t5_map(CUtensorMap* mp, const void* base, int64_t rows, int n, int64_t ld, int box_rows) {
    const auto fn = t5_encoder();
    if (!fn || !base || rows < 1 || rows > (int64_t)INT32_MAX) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(mp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
static bool t5_maps(const SrcCompress& s, int n, T5Maps& mp) {
    return t5_map(&mp.x0, s.c.A, s.c.rows_total, n, s.c.lda, 128);
}
// 8-row boxes stay inside one slab when k % 8 == 0
static bool t5_maps(const SrcQuery& s, int n, T5Maps& mp) {
    // ragged stacks: rows come through the row map, not in 8-row slab boxes
    if (s.a.k % 8 != 0 || s.a.rowmap) return false;
    if (!t5_map(&mp.x0, s.a.M, s.a.m_rows, n, n, 8)) return false;
    return s.a.wst ? t5_map(&mp.x1, s.a.wst, s.a.w_rows, n, n, 8) : t5_map(&mp.x1, s.a.M, s.a.m_rows, n, n, 8);
}

// Accuracy test of every item's factors, then refinement of the items that
// fail it (zs_certify.cuh).  The refinement needs n <= 512 (its basis and tiles
// in shared memory); above that a failing item is counted as not converged.
template <class Src, typename Tin>
static cudaError_t certify_launch(const Src& src, const TcScratch& sc, int n, int kw, int max_items, int num_sms,
                                  cudaStream_t st) {
    ZS_TRY(cudaMemsetAsync(sc.list, 0, 2 * sizeof(int), st));
    TcScratch scc = sc;
    scc.cplan = nullptr;
    {
        const size_t sm = ck_smem_bytes(n, kw, std::is_same<Tin, __nv_bfloat16>::value);
        int dev = 0, smem_sm = 0, resv = 0;
        ZS_TRY(cudaGetDevice(&dev));
        ZS_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        ZS_TRY(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
        const int per_sm = std::max(1, std::min(4, smem_sm / (int)(sm + 1024 + resv)));
        if constexpr (std::is_same<Src, SrcQuery>::value) {
            // stacked matrices cut into parts where a batch has too few queries
            // to balance the SMs by itself (measured: 0.76 -> 0.65 ms at 1,024
            // queries; at 4,096 and 20,000 queries the parts only cost); the
            // items' n x n scratch must hold n / kwp partial results
            if (max_items < 4 * num_sms * per_sm && n >= 2 * ((kw + 7) / 8 * 8)) {
                scc.cplan = sc.cplan;
                k_check_plan<Src><<<1, 1024, 0, st>>>(src, sc, n, kw);
                ZS_TRY(cudaGetLastError());
            }
        }
        // parts of stacked query matrices outnumber the items: a full persistent grid there
        const int grid = std::max(1, scc.cplan ? num_sms * per_sm : std::min(max_items, num_sms * per_sm));
        prof::Scope ps(std::is_same<Src, SrcQuery>::value ? "check_query" : "check", st);
        auto go = [&](auto kern) -> cudaError_t {
            ZS_TRY(set_smem(kern, sm));
            kern<<<grid, 256, sm, st>>>(src, scc, n, kw);
            return cudaGetLastError();
        };
        // 16-row tiles of R per warp: 1 (n <= 128), 2 (n <= 256), 4 (blocks of 512 columns)
        const int ntw = n <= 128 ? 1 : (n <= 256 ? 2 : 4);
        if (kw <= 16) {
            if (ntw == 1) ZS_TRY(go(k_check<Src, Tin, 1, 2>));
            else if (ntw == 2) ZS_TRY(go(k_check<Src, Tin, 2, 2>));
            else ZS_TRY(go(k_check<Src, Tin, 4, 2>));
        } else if (kw <= 32) {
            if (ntw == 1) ZS_TRY(go(k_check<Src, Tin, 1, 4>));
            else if (ntw == 2) ZS_TRY(go(k_check<Src, Tin, 2, 4>));
            else ZS_TRY(go(k_check<Src, Tin, 4, 4>));
        } else {
            if (ntw == 1) ZS_TRY(go(k_check<Src, Tin, 1, 8>));
            else if (ntw == 2) ZS_TRY(go(k_check<Src, Tin, 2, 8>));
            else ZS_TRY(go(k_check<Src, Tin, 4, 8>));
        }
    }
    {
        prof::Scope ps(std::is_same<Src, SrcQuery>::value ? "refine_query" : "refine", st);
        const int grid = std::max(1, std::min(max_items, num_sms));
        const size_t sm = rf_smem_bytes(n);
        if (n <= 256) {
            ZS_TRY(set_smem(k_refine<Src, Tin, 1>, sm));
            k_refine<Src, Tin, 1><<<grid, kRefineThreads, sm, st>>>(src, sc, n, kw);
        } else if (n <= 512) {
            ZS_TRY(set_smem(k_refine<Src, Tin, 2>, sm));
            k_refine<Src, Tin, 2><<<grid, kRefineThreads, sm, st>>>(src, sc, n, kw);
        } else {
            k_count_listed<<<1, 32, 0, st>>>(sc.list, sc.noconv);
        }
        ZS_TRY(cudaGetLastError());
    }
    note_launches(2);
    return cudaSuccess;
}

template <class Src, typename Tin, bool REF, bool QUERY>
static cudaError_t tc_core(const Src& src, TcScratch sc, int n, int kw, int max_items, int64_t max_tiles,
                           int ews_ctas, int num_sms, const Tuning& tu, cudaStream_t st, bool rows_aligned16) {
    // tcgen05 projection (TMA loads): the basis kernels also write Q~^T
    // (canonical layout) after Q~
    T5Maps maps;
    memset(&maps, 0, sizeof maps);
    const bool t5 = std::is_same<Tin, float>::value && tu.tc5_project && n % 32 == 0 && sc.m <= 64 &&
                    rows_aligned16 && t5_maps(src, n, maps);
    sc.Qt = t5 ? sc.Qf + (size_t)max_items * n * sc.m : nullptr;
    const int ntile = (n + 127) / 128;
    const int npairs = ntile * (ntile + 1) / 2;
    const int gi = std::min(max_items, 65535);
    const int proj_per_sm = tu.project_ctas_per_sm;
    if (tu.fused_sketch && sketch_fits(n, sc.m, QUERY)) {
        {
            prof::Scope ps(QUERY ? "sketch_query" : "sketch", st);
            ZS_TRY((sketch_dispatch<Src, Tin>(src, sc, n, max_items, st)));
        }
        {
            prof::Scope ps(QUERY ? "orth_query" : "orth", st);
            ZS_TRY((orth_dispatch<Src>(src, sc, n, max_items, st)));
        }
    } else {
        {
            prof::Scope ps(QUERY ? "gram_lo_query" : "gram_lo", st);
            k_gram_lo<Src, Tin><<<dim3(npairs, gi), 256, 0, st>>>(src, sc, n);
        }
        ZS_TRY(cudaGetLastError());
        bool yglob;
        const size_t sm = tc_subspace_smem(n, sc.m, yglob);
        const int gs = std::min(gi, yglob ? ews_ctas : 65535);
        prof::Scope ps(QUERY ? "subspace_query" : "subspace", st);
        if (sc.m <= 32) {
            ZS_TRY(set_smem(k_subspace<Src, 32>, sm));
            k_subspace<Src, 32><<<gs, 256, sm, st>>>(src, sc, n, yglob ? 1 : 0);
        } else {
            ZS_TRY(set_smem(k_subspace<Src, 64>, sm));
            k_subspace<Src, 64><<<gs, 256, sm, st>>>(src, sc, n, yglob ? 1 : 0);
        }
        ZS_TRY(cudaGetLastError());
    }
    if (t5) {
        // tcgen05 projection: as many CTAs per SM as the stage ring lets fit
        // (two for m <= 32; TMEM: 256 columns each)
        const size_t sm = t5_smem_bytes(sc.m);
        ZS_TRY(set_smem(k_project_tc5<Src>, sm));
        ZS_TRY(cudaFuncSetAttribute(k_project_tc5<Src>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared));
        prof::Scope ps(QUERY ? "project_query" : "project", st);
        // CTAs per SM: shared memory (with the per-block reservation) and TMEM
        // (512 columns per SM); registers (< 128 per thread) are not binding
        int dev = 0, smem_sm = 0, resv = 0;
        ZS_TRY(cudaGetDevice(&dev));
        ZS_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        ZS_TRY(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
        const int per_sm = std::max(1, std::min(smem_sm / (int)(sm + resv), (int)(512 / kT5Cols)));
        const int gp = (int)std::min<int64_t>(max_tiles, (int64_t)num_sms * per_sm);
        k_project_tc5<Src><<<std::max(gp, 1), kT5Threads, sm, st>>>(src, sc, n, maps);
    } else {
        const size_t sm = project_smem_bytes(sc.m);
        ZS_TRY(set_smem(k_project<Src, Tin>, sm));
        prof::Scope ps(QUERY ? "project_query" : "project", st);
        const int gp = (int)std::min<int64_t>(max_tiles, (int64_t)num_sms * proj_per_sm);
        k_project<Src, Tin><<<std::max(gp, 1), 256, sm, st>>>(src, sc, n);
    }
    ZS_TRY(cudaGetLastError());
    if (!REF && sc.m <= 32) {
        prof::Scope ps(QUERY ? "rr_core_query" : "rr_core", st);
        k_rr_core_reg<Src><<<(max_items + 3) / 4, 128, 0, st>>>(src, sc, kw);
    } else {
        // one item per CTA: the Jacobi rounds' rotations and the small
        // products spread over 128 threads (one warp per item left the FP64
        // refinement and the m > 32 sweeps latency-bound)
        const size_t sm = rr_warp_bytes<REF>(sc.m);
        ZS_TRY(set_smem(k_rr_core<Src, REF>, sm));
        prof::Scope ps(QUERY ? "rr_core_query" : "rr_core", st);
        k_rr_core<Src, REF><<<std::min(max_items, 65535), 128, sm, st>>>(src, sc, kw);
    }
    ZS_TRY(cudaGetLastError());
    {
        const size_t sm = rr_out_smem_bytes(n, sc.m, kw);
        ZS_TRY(set_smem(k_rr_out<Src, QUERY>, sm));
        prof::Scope ps(QUERY ? "rr_out_query" : "rr_out", st);
        k_rr_out<Src, QUERY><<<gi, 256, sm, st>>>(src, sc, n, kw);
    }
    ZS_TRY(cudaGetLastError());
    ZS_TRY((certify_launch<Src, Tin>(src, sc, n, kw, max_items, num_sms, st)));
    note_launches(5);
    return cudaSuccess;
}

template <typename T, int KMAX, int QMAX>
static void lift_launch(const QueryArgs& a, int64_t max_slabs, int num_sms, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        // tensor-core lift: per warp two split copies of C in shared memory
        const int threads = (KMAX * QMAX >= 2048) ? 128 : 256;
        const int wpc = threads / 32;
        const int grid =
            (int)std::max<int64_t>(1, std::min<int64_t>((max_slabs + wpc - 1) / wpc, (int64_t)num_sms * 8));
        if (a.k % 16 == 0) {
            const size_t sm = sizeof(float) * lift_tc_warp_floats<KMAX, QMAX>() * wpc;
            set_smem(k_lift_tc<KMAX, QMAX>, sm);
            k_lift_tc<KMAX, QMAX><<<grid, threads, sm, st>>>(a);
        } else {
            const size_t sm = sizeof(float) * lift_nat_warp_floats<KMAX, QMAX>() * wpc;
            set_smem(k_lift_tc_nat<KMAX, QMAX>, sm);
            k_lift_tc_nat<KMAX, QMAX><<<grid, threads, sm, st>>>(a);
        }
    } else {
        const int threads = (KMAX * QMAX >= 2048) ? 128 : 256;       // register budget
        const int wpc = threads / 32;
        const size_t sm = sizeof(T) * (size_t)KMAX * QMAX * wpc;
        set_smem(k_lift<T, KMAX, QMAX>, sm);
        const int grid =
            (int)std::max<int64_t>(1, std::min<int64_t>((max_slabs + wpc - 1) / wpc, (int64_t)num_sms * 8));
        k_lift<T, KMAX, QMAX><<<grid, threads, sm, st>>>(a);
    }
}

template <typename T, int KMAX>
static void lift_q(const QueryArgs& a, int64_t max_slabs, int num_sms, cudaStream_t st) {
    // the output width k_out (zero columns past k_q included) selects QMAX
    if (a.kout <= 16) lift_launch<T, KMAX, 16>(a, max_slabs, num_sms, st);
    else if (a.kout <= 32) lift_launch<T, KMAX, 32>(a, max_slabs, num_sms, st);
    else lift_launch<T, KMAX, 64>(a, max_slabs, num_sms, st);
}

template <typename T>
static cudaError_t launch_lift(const QueryArgs& a, int64_t max_slabs, int num_sms, cudaStream_t st) {
    prof::Scope ps("lift", st);
    if (a.k <= 16) lift_q<T, 16>(a, max_slabs, num_sms, st);
    else if (a.k <= 32) lift_q<T, 32>(a, max_slabs, num_sms, st);
    else lift_q<T, 64>(a, max_slabs, num_sms, st);
    return cudaGetLastError();
}

template <typename T, bool REF>
static cudaError_t query_impl(const QueryArgs& a, const QueryGrid& g, int flags, const Tuning& tu, int num_sms,
                              cudaStream_t st) {
    const int max_nq = g.nq;
    const int64_t max_slabs = g.slabs;
    const bool fp64 = std::is_same<T, double>::value;
    const int k = a.k, n = a.n, kq = a.kq;
    const int pers = std::max(1, num_sms * tu.slab_ctas_per_sm);
    const bool tc = use_tc_path(fp64, n, flags);
    // Partial-SVD
    {
        const int ld = k + 1;
        auto r16 = [](size_t b) { return (b + 15) & ~size_t(15); };
        size_t sm = 2 * r16(sizeof(T) * k * ld) + r16(sizeof(T) * 64 * ld);
        if (REF) sm += 3 * r16(sizeof(double) * k * ld);
        prof::Scope ps("partial_svd", st);
        if (std::is_same<T, float>::value && !REF && k <= 32) {
            // one warp per boundary slab (2 per query), 4 warps per CTA
            if (k <= 16) k_partial_warp<16><<<(2 * max_nq + 3) / 4, 128, 0, st>>>(a);
            else k_partial_warp<32><<<(2 * max_nq + 3) / 4, 128, 0, st>>>(a);
        } else {
            ZS_TRY(set_smem(k_partial<T, REF>, sm));
            k_partial<T, REF><<<std::min(2 * max_nq, pers), 256, sm, st>>>(a);
        }
        ZS_TRY(cudaGetLastError());
    }
    if (!(tc && a.wst)) {      // interior slabs are read in place from the store's Sigma V^T otherwise
        prof::Scope ps("stack", st);
        k_stack<T><<<(int)std::min<int64_t>(max_slabs, pers), 256, 0, st>>>(a);
        ZS_TRY(cudaGetLastError());
        note_launches(1);
    }
    if constexpr (!std::is_same<T, double>::value) {
        if (tc) {
            TcScratch sc;
            sc.G = (float*)a.G;
            sc.Qf = (float*)a.qb;
            sc.Y = (float*)a.ys;
            sc.ews = a.ews;
            sc.ews_ctas = std::max(1, a.ews_ctas);
            sc.m = tc_width(kq, tu.eig_m_extra);
            sc.power_its = tu.power_its;
            tc_aux_carve(a.aux, max_nq, a.aux_tiles, sc.m, kq, sc);
            sc.fault = a.fault;
            sc.noconv = a.noconv;
            sc.refined = a.refined;
            sc.xi = 0.0;
            sc.energy = nullptr;
            sc.kxi = nullptr;
            SrcQuery src{a};
            if (a.rowmap) {
                prof::Scope ps("ragged_map", st);
                k_ragged_prefix<<<1, 1024, 0, st>>>(a);
                k_ragged_map<<<std::min(max_nq, pers), 256, 0, st>>>(a);
                ZS_TRY(cudaGetLastError());
                note_launches(2);
            }
            // stacked rows (M and the store's Sigma V^T) are 16-byte aligned when n % 4 == 0
            ZS_TRY((tc_core<SrcQuery, float, REF, true>(src, sc, n, kq, max_nq, g.tiles, sc.ews_ctas, num_sms,
                                                        tu, st, n % 4 == 0)));
            if (a.rowmap) {
                prof::Scope ps("ragged_expand", st);
                k_ragged_expand<<<std::min(max_nq, pers), 256, 0, st>>>(a);
                ZS_TRY(cudaGetLastError());
                note_launches(1);
            }
            {
                const size_t sm = sizeof(float) * ((size_t)k * k + (size_t)k * kq);
                ZS_TRY(set_smem(k_bfix, sm));
                prof::Scope ps("boundary_fix", st);
                k_bfix<<<std::min(2 * max_nq, pers), 256, sm, st>>>(a);
                ZS_TRY(cudaGetLastError());
            }
            if (a.lift) ZS_TRY(launch_lift<T>(a, max_slabs, num_sms, st));
            note_launches(a.lift ? 3 : 2);
            return cudaSuccess;
        }
    }
    {
        const int ntile = (n + 63) / 64;
        const int npairs = ntile * (ntile + 1) / 2;
        dim3 gg(npairs, std::min(max_nq, 65535));
        prof::Scope ps("gram_query", st);
        k_gram_query<T><<<gg, 256, 0, st>>>(a);
        ZS_TRY(cudaGetLastError());
    }
    {
        const EigPlan ep = eig_plan(n, kq, tu.eig_m_extra, fp64, REF);
        if (!ep.ok) return cudaErrorInvalidValue;
        const int grid = std::min(max_nq, ep.yglob ? a.ews_ctas : 65535);
        if (ep.m <= 32) {
            ZS_TRY(set_smem(k_eig_query<T, REF, 32>, ep.smem));
            prof::Scope ps("eig_query", st);
            k_eig_query<T, REF, 32><<<grid, 256, ep.smem, st>>>(a, ep.m, ep.yglob, a.ews);
        } else {
            ZS_TRY(set_smem(k_eig_query<T, REF, 64>, ep.smem));
            prof::Scope ps("eig_query", st);
            k_eig_query<T, REF, 64><<<grid, 256, ep.smem, st>>>(a, ep.m, ep.yglob, a.ews);
        }
        ZS_TRY(cudaGetLastError());
    }
    {
        const size_t sm = sizeof(T) * ((size_t)kq * (n + 1) + (size_t)k * (n + 1) + (size_t)k * kq + (size_t)k * k) + 64;
        ZS_TRY(set_smem(k_ur<T>, sm));
        prof::Scope ps("stitched_u", st);
        k_ur<T><<<std::min(max_nq, pers), 256, sm, st>>>(a);
        ZS_TRY(cudaGetLastError());
    }
    if (a.lift) ZS_TRY(launch_lift<T>(a, max_slabs, num_sms, st));
    note_launches(a.lift ? 5 : 4);
    return cudaSuccess;
}

// Per-precision query launchers (zs_query_f64.cu, zs_query_f32.cu, zs_query_f32r.cu).
cudaError_t launch_query_f64(const QueryArgs& a, const QueryGrid& g, int flags, const Tuning& tu, int num_sms,
                             cudaStream_t st);
cudaError_t launch_query_f32(const QueryArgs& a, const QueryGrid& g, int flags, const Tuning& tu, int num_sms,
                             cudaStream_t st);
cudaError_t launch_query_f32_refine(const QueryArgs& a, const QueryGrid& g, int flags, const Tuning& tu,
                                    int num_sms, cudaStream_t st);
cudaError_t launch_compress_simt(const CompressChunk& c, bool fp64, int flags, const Tuning& tu, int num_sms,
                                 cudaStream_t st);
cudaError_t launch_compress_tc(const CompressChunk& c, int flags, const Tuning& tu, int num_sms, cudaStream_t st);

}  // namespace zs
