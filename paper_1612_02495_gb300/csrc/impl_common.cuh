// Launch wrappers shared by the per-scheme translation units.
#pragma once
#include <string.h>

#include <type_traits>

#include "impl.h"
#include "kernels.cuh"

namespace swept {

template <typename T, class Op>
struct Launch {
  static typename Op::K kc(const void* k) {
    typename Op::K kk;
    memcpy(&kk, k, sizeof(kk));
    return kk;
  }
  static int64_t smem_values(int M) { return swept_smem_values<Op>(M); }
  // register tiers exist for scalar schemes
  static constexpr bool p_ok(int P) { return P == 0 || Op::C == 1; }
  // fn(std::integral_constant<int, P>) for the kernel variant of g.P
  template <class Fn>
  static cudaError_t with_p(int P, Fn&& fn) {
    switch (P) {
      case 0: return fn(std::integral_constant<int, 0>{});
      case 1: if constexpr (p_ok(1)) return fn(std::integral_constant<int, 1>{}); break;
      case 2: if constexpr (p_ok(2)) return fn(std::integral_constant<int, 2>{}); break;
      case 4: if constexpr (p_ok(4)) return fn(std::integral_constant<int, 4>{}); break;
      case 8: if constexpr (p_ok(8)) return fn(std::integral_constant<int, 8>{}); break;
      default: break;
    }
    return cudaErrorInvalidValue;
  }
  // The shared-memory-tier kernels also exist with 256-thread launch bounds (up
  // to 85 registers a thread instead of 64), used whenever a block has <= 256
  // threads: measured faster for Euler (no flux-phase spills) and slightly for KS
  static constexpr bool kSmallBlockVariant = true;
  // fn(std::integral_constant<int, MAXT>) for the launch-bounds variant of (P, threads);
  // the 256-thread variant exists only for tiers in shared memory (P = 0)
  template <int P, class Fn>
  static cudaError_t with_maxt(int threads, Fn&& fn) {
    if constexpr (kSmallBlockVariant && P == 0) {
      if (threads <= 256) return fn(std::integral_constant<int, 256>{});
    }
    return fn(std::integral_constant<int, 1024>{});
  }
  static cudaError_t prepare(size_t bytes) {
    cudaError_t e = raise_smem_limit((const void*)k_swept_up<T, Op>, bytes);
    if (e == cudaSuccess) e = raise_smem_limit((const void*)k_swept_diamond<T, Op>, bytes);
    if constexpr (kSmallBlockVariant) {
      if (e == cudaSuccess) e = raise_smem_limit((const void*)k_swept_up<T, Op, 0, 256>, bytes);
      if (e == cudaSuccess) e = raise_smem_limit((const void*)k_swept_diamond<T, Op, 0, 256>, bytes);
    }
    return e;
  }
  static cudaError_t up(const Geom& g, const void* k, const void* u_in, void* u_out, void* e_out, int hh,
                        int write_top, int threads, size_t smem, cudaStream_t s) {
    return with_p(g.P, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      return with_maxt<P>(threads, [&](auto mc) {
        constexpr int MAXT = decltype(mc)::value;
        k_swept_up<T, Op, P, MAXT><<<(unsigned)g.nt, threads, smem, s>>>(g, kc(k), (const T*)u_in, (T*)u_out,
                                                                         (T*)e_out, hh, write_top);
        return cudaGetLastError();
      });
    });
  }
  static cudaError_t diamond(const Geom& g, const void* k, void* u_out, const void* e_in, void* e_out, int odd,
                             int mode, int hh, int threads, size_t smem, cudaStream_t s) {
    return with_p(g.P, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      return with_maxt<P>(threads, [&](auto mc) {
        constexpr int MAXT = decltype(mc)::value;
        k_swept_diamond<T, Op, P, MAXT><<<(unsigned)g.nt, threads, smem, s>>>(g, kc(k), (T*)u_out, (const T*)e_in,
                                                                              (T*)e_out, odd, mode, hh);
        return cudaGetLastError();
      });
    });
  }
  static cudaError_t classic(const Geom& g, const void* k, int stage, const void* in, void* out, cudaStream_t s) {
    const int B = 256;
    const unsigned grid = (unsigned)((g.N + B - 1) / B);
    if (stage == 0)
      k_classic<T, Op, 0><<<grid, B, 0, s>>>(g.N, g.bc, kc(k), (const T*)in, (T*)out);
    else
      k_classic<T, Op, 1><<<grid, B, 0, s>>>(g.N, g.bc, kc(k), (const T*)in, (T*)out);
    return cudaGetLastError();
  }
  static cudaError_t copy(int64_t n, const void* src, void* dst, cudaStream_t s) {
    k_copy<T><<<1024, 256, 0, s>>>(n, (const T*)src, (T*)dst);
    return cudaGetLastError();
  }
  static cudaError_t persist(const Geom& g, const void* k, void* u, void* e0, void* e1, int64_t n_sub, int* done,
                             unsigned long long* queue, int* error, uint32_t spin_limit, int64_t start_item,
                             int blocks, int threads, size_t smem, cudaStream_t s) {
    return with_p(g.P, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      return with_maxt<P>(threads, [&](auto mc) {
        constexpr int MAXT = decltype(mc)::value;
        cudaError_t e = raise_smem_limit((const void*)k_swept_persist<T, Op, P, MAXT>, smem);
        if (e != cudaSuccess) return e;
        PersistCtl c{done, queue, error, spin_limit, start_item};
        k_swept_persist<T, Op, P, MAXT><<<blocks, threads, smem, s>>>(g, kc(k), (T*)u, (T*)e0, (T*)e1, n_sub, c);
        return cudaGetLastError();
      });
    });
  }
  static int persist_blocks_per_sm(int P_, int threads, size_t smem) {
    int n = 0;
    const cudaError_t e = with_p(P_, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      return with_maxt<P>(threads, [&](auto mc) {
        constexpr int MAXT = decltype(mc)::value;
        cudaError_t e2 = raise_smem_limit((const void*)k_swept_persist<T, Op, P, MAXT>, smem);
        if (e2 != cudaSuccess) return e2;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_swept_persist<T, Op, P, MAXT>, threads, smem);
      });
    });
    return e == cudaSuccess ? n : 0;
  }
  // smem = window bytes; the two export areas (2 E values) are added here
  static cudaError_t cluster(const Geom& g, const void* k, void* u, int64_t n_sub, int threads, size_t smem,
                             cudaStream_t s) {
    return with_p(g.P, [&](auto pc) { return cluster_p<decltype(pc)::value>(g, k, u, n_sub, threads, smem, s); });
  }
  template <int P>
  static cudaError_t cluster_p(const Geom& g, const void* k, void* u, int64_t n_sub, int threads, size_t smem,
                               cudaStream_t s) {
    const int64_t win_values = (int64_t)(smem / sizeof(T));
    const size_t bytes = smem + 2 * (size_t)g.E * sizeof(T);
    auto fn = k_swept_cluster<T, Op, P>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = raise_smem_limit((const void*)fn, bytes);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g.nt, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)g.nt;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, g, kc(k), (T*)u, n_sub, win_values);
  }
  static cudaError_t slab_prepare(size_t bytes) {
    cudaError_t e = raise_smem_limit((const void*)k_slab_up<T, Op>, bytes);
    if (e == cudaSuccess) e = raise_smem_limit((const void*)k_slab_diamond<T, Op>, bytes);
    return e;
  }
  static cudaError_t slab_up(const Geom& g, const Slab& sl, const void* k, const void* u_in, void* u_out, void* e_out,
                             int hh, int write_top, int threads, size_t smem, cudaStream_t s) {
    return with_p(g.P, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      k_slab_up<T, Op, P><<<(unsigned)sl.nb, threads, smem, s>>>(g, sl, kc(k), (const T*)u_in, (T*)u_out,
                                                                  (T*)e_out, hh, write_top);
      return cudaGetLastError();
    });
  }
  static cudaError_t slab_diamond(const Geom& g, const Slab& sl, const void* k, void* u_out, const void* e_in,
                                  void* e_out, int odd, int mode, int hh, int threads, size_t smem, cudaStream_t s) {
    return with_p(g.P, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      k_slab_diamond<T, Op, P><<<(unsigned)sl.nb, threads, smem, s>>>(g, sl, kc(k), (T*)u_out, (const T*)e_in,
                                                                       (T*)e_out, odd, mode, hh);
      return cudaGetLastError();
    });
  }
  static Tape<T> mk_tape(void* tape, int64_t tier0, int64_t ntiers, int64_t base) {
    Tape<T> t;
    t.p = (T*)tape;
    t.tier0 = tier0;
    t.ntiers = ntiers;
    t.base = base;
    return t;
  }
  static cudaError_t prepare_tape(size_t bytes) {
    cudaError_t e = raise_smem_limit((const void*)k_swept_up_tape<T, Op>, bytes);
    if (e != cudaSuccess) return e;
    return raise_smem_limit((const void*)k_swept_diamond_tape<T, Op>, bytes);
  }
  static cudaError_t up_tape(const Geom& g, const void* k, const void* u_in, void* u_out, void* e_out, int hh,
                             int write_top, int threads, size_t smem, void* tape, int64_t tier0, int64_t ntiers,
                             int64_t base, cudaStream_t s) {
    if (smem > 48 * 1024) {
      cudaError_t e = prepare_tape(smem);
      if (e != cudaSuccess) return e;
    }
    k_swept_up_tape<T, Op><<<(unsigned)g.nt, threads, smem, s>>>(g, kc(k), (const T*)u_in, (T*)u_out, (T*)e_out, hh,
                                                                 write_top, mk_tape(tape, tier0, ntiers, base));
    return cudaGetLastError();
  }
  static cudaError_t diamond_tape(const Geom& g, const void* k, void* u_out, const void* e_in, void* e_out, int odd,
                                  int mode, int hh, int threads, size_t smem, void* tape, int64_t tier0,
                                  int64_t ntiers, int64_t base, cudaStream_t s) {
    if (smem > 48 * 1024) {
      cudaError_t e = prepare_tape(smem);
      if (e != cudaSuccess) return e;
    }
    k_swept_diamond_tape<T, Op><<<(unsigned)g.nt, threads, smem, s>>>(
        g, kc(k), (T*)u_out, (const T*)e_in, (T*)e_out, odd, mode, hh, mk_tape(tape, tier0, ntiers, base));
    return cudaGetLastError();
  }
};

// launch wrappers of the adjoint passes for adjoint operator AOp
template <typename T, class AOp>
struct AdjLaunch {
  static typename AOp::K kc(const void* k) {
    typename AOp::K kk;
    memcpy(&kk, k, sizeof(kk));
    return kk;
  }
  static cudaError_t prepare(size_t bytes) {
    cudaError_t e = raise_smem_limit((const void*)k_adj_up<T, AOp>, bytes);
    if (e != cudaSuccess) return e;
    return raise_smem_limit((const void*)k_adj_diamond<T, AOp>, bytes);
  }
  static cudaError_t up(const Geom& g, const void* ka, const void* lam_in, void* lam_out, void* e_out, int hh,
                        int write_top, int threads, size_t smem, const void* tape, int64_t top, int64_t base,
                        double* slots, cudaStream_t s) {
    k_adj_up<T, AOp><<<(unsigned)g.nt, threads, smem, s>>>(g, kc(ka), (const T*)lam_in, (T*)lam_out, (T*)e_out, hh,
                                                           write_top, (const T*)tape, top, base, slots);
    return cudaGetLastError();
  }
  static cudaError_t diamond(const Geom& g, const void* ka, void* lam_out, const void* e_in, void* e_out, int odd,
                             int mode, int hh, int threads, size_t smem, const void* tape, int64_t top, int64_t base,
                             double* slots, cudaStream_t s) {
    k_adj_diamond<T, AOp><<<(unsigned)g.nt, threads, smem, s>>>(g, kc(ka), (T*)lam_out, (const T*)e_in, (T*)e_out,
                                                                odd, mode, hh, (const T*)tape, top, base, slots);
    return cudaGetLastError();
  }
};

}  // namespace swept
