// Device engine for one block size B and one V-cycle precision:
//   T  = float64 or float32 (V-cycle matrices and vectors),
//   TD = storage type of the smoother block inverses (T or bfloat16).
// The outer PCG (Section 6) is always float64 on the float64 fine operator.
//
// Solver graphs: the PCG set-up kernels, then a CUDA-graph WHILE node whose
// body is one PCG iteration; the convergence test in k_cg_update ends the
// loop on the device, so a whole solve (or time step) is one graph launch
// with no host round trip. If the runtime refuses conditional nodes, the
// engine falls back to launching the iteration graph in batches and polling
// the device flag.
#pragma once
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/aggmg.h"
#include "cg_kernels.cuh"
#include "engine.h"
#include "kernels.cuh"
#include "face_op.cuh"
#include "mf_kernels.cuh"
#include "coarse_kernels.cuh"
#include "coarse_persistent.cuh"

namespace aggmg {

#define AGG_CK(call)                                                              \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      err = std::string(#call) + " failed: " + cudaGetErrorString(e_);            \
      return AGG_ECUDA;                                                           \
    }                                                                             \
  } while (0)

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename TS>
inline TS to_storage(double v) {
  return static_cast<TS>(v);
}
template <>
inline __nv_bfloat16 to_storage<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}

template <typename T, typename TD, int B>
class Engine : public EngineBase {
  static constexpr int NTB = UnitThreads<B>::value;
  static constexpr bool kRL = (B <= 32);
#ifndef AGG_COARSE_NT
#define AGG_COARSE_NT 256
#endif
  // threads per block of the coarsest triangular products (one warp per row;
  // 64 measured no faster than 256)
  static constexpr int kCoarseNT = AGG_COARSE_NT;
  // coarse levels on the row-lane kernels: warp-shuffle units (B <= 32, kRL;
  // also eligible for the persistent and cluster kernels) or shared-memory
  // units (B = 64)
  static constexpr bool kRowLanes = kRL || B == 64;
  // matrix-free fine operator: float32 V-cycle on quadrilaterals of p = 1..3
  // and hexahedra of p = 1, 2
  static constexpr bool kMf =
      std::is_same<T, float>::value && (B == 4 || B == 9 || B == 16 || B == 8 || B == 27 || B == 64);
  using MfOpT = typename std::conditional<kMf, typename MfOpFor<kMf ? B : 9>::type, SellOp<T, B>>::type;
  bool mf_ = false;
  MfOpT mfop_{};
  int64_t mf_bytes_ = 0;
  // float64 matrix-free level-0 operator (a measured alternative to the
  // face-structured float64 operator of the outer CG; built on first use)
  static constexpr bool kMf64 = (B == 4 || B == 9 || B == 16 || B == 8 || B == 27);
  using Mf64T = typename std::conditional<kMf64, typename MfOpForT<double, kMf64 ? B : 9>::type,
                                          SellOp<double, B>>::type;
  Mf64T mf64_{};
  bool mf64_ready_ = false;
  int64_t mf64_bytes_ = 0;
  const Mesh* mesh_ = nullptr;
  std::vector<int64_t> perm0_, inv0_;
  double mass_coeff_ = 0.0;
  struct Lev {
    int64_t n = 0, nsl = 0, nvec = 0;
    int32_t* slice_ptr = nullptr;
    int32_t* cols = nullptr;
    T* vals = nullptr;
    TD* Dinv = nullptr;
    T* P = nullptr;
    int32_t* parent = nullptr;
    int64_t* child_ptr = nullptr;
    int64_t* perm = nullptr;
    T *xa = nullptr, *xb = nullptr, *d = nullptr, *rhs = nullptr, *S = nullptr;
    std::vector<T> c1, c2;
    // row-lane copies for levels >= 1 (column-major blocks)
    CsrBlocks<T> rl{};
    TD* rl_dinv = nullptr;
    T* rl_P = nullptr;
    SellView<T> A() const { return SellView<T>{slice_ptr, cols, vals, nsl}; }
  };

  std::vector<Lev> lev_;
  std::vector<int64_t> nnzb_;
  int num_sms_ = 152;
  // persistent kernel for levels >= 1 and the coarsest solve (row-lane
  // levels, at least one smoothed coarse level), when asked for
  bool persist_ = false;
  GridBar* bar_ = nullptr;
  PCoarse<T, TD> pc_{};
  int pgrid_ = 0;
  // thread-block cluster kernel for the smallest levels (from lc_ on, each of
  // at most csize_ x CNT rows) and the coarsest solve
  bool cluster_ = false;
  int lc_ = 0, csize_ = 0;
  PCoarse<T, TD> pcc_{};

  // Grid of a slice-looping unit kernel: one slice per warp. (Sizing the grid
  // to the resident warps and looping removes the partial last wave, but the
  // lower concurrency cost more bandwidth than the tail saved on GB300.)
  template <typename K>
  int64_t bgrid(K, int64_t nsl) const {
    return std::max<int64_t>(1, cdiv(nsl * SL, NTB));
  }
  int nlev_ = 0, degree_ = 3;

  // float64 quadrature data of the matrix-free operator (first use only)
  int build_mf64(std::string& err) {
    if (mf64_ready_) return AGG_OK;
    if constexpr (!kMf64) {
      err = "the float64 matrix-free operator needs quadrilaterals of p <= 3 or hexahedra of p <= 2";
      return AGG_EUNSUPPORTED;
    } else {
      MatrixFreeData md;
      int rc;
      if ((rc = matrix_free_build(*mesh_, perm0_, inv0_, mass_coeff_, md, err))) return rc;
      if (md.q != Mf64T::kDegree + 2) { err = "matrix-free operator needs quad_extra = 1"; return AGG_EUNSUPPORTED; }
      double *cell, *face;
      int32_t* nbr;
      int8_t* code;
      if ((rc = upload(&cell, md.cell.data(), md.cell.size(), err))) return rc;
      if ((rc = upload(&face, md.face.data(), md.face.size(), err))) return rc;
      if ((rc = upload(&nbr, md.nbr.data(), md.nbr.size(), err))) return rc;
      if ((rc = upload(&code, md.code.data(), md.code.size(), err))) return rc;
      mf64_.V = MfViewT<double>{cell, face, nbr, code, lev_[0].nsl};
      Tables1D t1 = make_tables(mesh_->p, md.q);
      std::memset(&mf64_.T, 0, sizeof(mf64_.T));
      for (int a = 0; a <= mesh_->p; ++a) {
        for (int kq = 0; kq < md.q; ++kq) {
          double v[8], dv[8];
          lagrange_eval(t1.gll.data(), mesh_->p + 1, t1.gx[kq], v, dv);
          mf64_.T.L[a][kq] = v[a];
          mf64_.T.D[a][kq] = dv[a];
        }
        for (int sd = 0; sd < 2; ++sd) {
          double v[8], dv[8];
          lagrange_eval(t1.gll.data(), mesh_->p + 1, (double)sd, v, dv);
          mf64_.T.Dend[sd][a] = dv[a];
        }
      }
      mf64_bytes_ = (int64_t)(md.cell.size() * 8 + md.face.size() * 8 + md.nbr.size() * 4 + md.code.size());
      mf64_ready_ = true;
      return AGG_OK;
    }
  }
  // level 0 in face-structured form: float64 for the outer CG, and the
  // V-cycle precision copy for the assembled smoother (the same data when
  // the V-cycle is float64)
  using A0Op = FaceOp<double, B>;
  using L0Op = FaceOp<T, B>;
  A0Op A0f_{};
  L0Op fop_{};
  double face_entries_ = 0;          // stored operator entries of level 0
  SellView<double> A0_{};            // slot structure of level 0 (adjoint face data), no values
  double* Me_ = nullptr;
  double *Linv_ = nullptr, *U_ = nullptr, *yc_ = nullptr;
  int64_t nc_ = 0;
  double *b_ = nullptr, *x_ = nullptr, *r_ = nullptr, *p_ = nullptr, *q_ = nullptr, *z_ = nullptr;
  double* partials_ = nullptr;
  float* r32_ = nullptr;
  CGState* st_ = nullptr;
  CGState* st_host_ = nullptr;
  std::vector<void*> allocs_;
  cudaStream_t cs_ = nullptr;
  bool use_cond_ = false;
  // solve graphs
  cudaGraphExec_t solve_exec_ = nullptr, init_exec_ = nullptr, body_exec_ = nullptr;
  std::vector<cudaGraph_t> graphs_;
  // simulation
  bool sim_ = false;
  SimParams sp_{};
  double *w_ = nullptr, *mask_ = nullptr;
  int64_t* step_ = nullptr;
  int *iters_ = nullptr, *slot_ = nullptr, *sim_status_ = nullptr;
  int cap_ = 1024;
  // adjoint data and buffers
  double *Ke_ = nullptr, *Y_ = nullptr;
  // BDF2 history and inverse element mass blocks
  double *up_ = nullptr, *wp_ = nullptr, *Minv_ = nullptr;
  bool hist_valid_ = false;
  std::vector<double> me_int_;     // element mass blocks, internal order (for M^-1)
  double *ua_ = nullptr, *wa_ = nullptr, *ub_ = nullptr, *wb_ = nullptr;
  cudaGraphExec_t step_exec_ = nullptr, step_pro_exec_ = nullptr, step_epi_exec_ = nullptr;

  template <typename X>
  int dalloc(X** p, size_t count, std::string& err) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(X));
    if (e != cudaSuccess) {
      err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      return AGG_ENOMEM;
    }
    cudaMemset(v, 0, std::max<size_t>(count, 1) * sizeof(X));
    allocs_.push_back(v);
    *p = static_cast<X*>(v);
    return AGG_OK;
  }
  template <typename X>
  int upload(X** p, const X* host, size_t count, std::string& err) {
    int s = dalloc(p, count, err);
    if (s) return s;
    AGG_CK(cudaMemcpy(*p, host, count * sizeof(X), cudaMemcpyHostToDevice));
    return AGG_OK;
  }

  // pack B x B row-major blocks into the sliced layout [k/VW][lane][k%VW], k = c*B + r
  template <typename TS>
  static void pack(const double* blk, TS* slot_base, int lane) {
    constexpr int VW = Vec<TS>::W;
    for (int k = 0; k < B * B; ++k) {
      const int c = k / B, r = k % B;
      slot_base[((size_t)(k / VW) * SL + lane) * VW + (k % VW)] = to_storage<TS>(blk[r * B + c]);
    }
  }

  template <typename TS>
  int upload_sell(const BlockCSR& A, int64_t nsl, int32_t** sp, int32_t** cols, TS** vals, std::string& err,
                  bool with_vals = true) {
    constexpr int KP = Pad<TS, B>::KP;
    const int64_t n = A.nrows;
    std::vector<int32_t> hsp(nsl + 1, 0);
    for (int64_t s = 0; s < nsl; ++s) {
      int64_t mx = 1;
      for (int64_t u = s * SL; u < std::min<int64_t>(n, (s + 1) * SL); ++u)
        mx = std::max<int64_t>(mx, A.rowptr[u + 1] - A.rowptr[u]);
      hsp[s + 1] = hsp[s] + (int32_t)mx;
    }
    const int64_t nslots = hsp[nsl];
    std::vector<int32_t> hc((size_t)nslots * SL, 0);
    std::vector<TS> hv(with_vals ? (size_t)nslots * SL * KP : 0, to_storage<TS>(0.0));
    for (int64_t s = 0; s < nsl; ++s)
      for (int lane = 0; lane < SL; ++lane) {
        const int64_t u = s * SL + lane;
        const int64_t len = (u < n) ? A.rowptr[u + 1] - A.rowptr[u] : 0;
        for (int64_t j = 0; j < hsp[s + 1] - hsp[s]; ++j) {
          const int64_t slot = hsp[s] + j;
          if (j < len) {
            const int64_t k = A.rowptr[u] + j;
            hc[slot * SL + lane] = A.col[k];
            if (with_vals) pack<TS>(&A.val[(size_t)k * B * B], &hv[(size_t)slot * SL * KP], lane);
          } else {
            hc[slot * SL + lane] = (int32_t)(u < n ? u : 0);
          }
        }
      }
    int s = upload(sp, hsp.data(), hsp.size(), err);
    if (!s) s = upload(cols, hc.data(), hc.size(), err);
    if (!s && with_vals) s = upload(vals, hv.data(), hv.size(), err);
    return s;
  }

  // smoother block inverses in the unit kernels' layout: packed upper
  // triangle of the symmetrised block for B <= 32, full blocks otherwise
  int upload_dinv(const std::vector<double>& blocks, int64_t n, int64_t nsl, TD** out, std::string& err) {
    if constexpr (B > 32) {
      return upload_blocks<TD>(blocks, n, nsl, out, err);
    } else {
      constexpr int KP = SymPad<TD, B>::KP, VW = Vec<TD>::W;
      std::vector<TD> hv((size_t)nsl * SL * KP, to_storage<TD>(0.0));
      for (int64_t u = 0; u < n; ++u) {
        const double* m = &blocks[(size_t)u * B * B];
        TD* sb = &hv[(size_t)(u / SL) * SL * KP];
        const int lane = (int)(u % SL);
        for (int j = 0; j < B; ++j)
          for (int i = 0; i <= j; ++i) {
            const int k = j * (j + 1) / 2 + i;
            sb[((size_t)(k / VW) * SL + lane) * VW + (k % VW)] = to_storage<TD>(0.5 * (m[i * B + j] + m[j * B + i]));
          }
      }
      return upload(out, hv.data(), hv.size(), err);
    }
  }

  // ROWS x COLS row-major block -> sliced column-major chunks (k = c ROWS + r)
  template <typename TS>
  static void pack_rect(const double* blk, TS* slot_base, int lane, int rows, int cols) {
    constexpr int VW = Vec<TS>::W;
    for (int k = 0; k < rows * cols; ++k) {
      const int c = k / rows, r = k % rows;
      slot_base[((size_t)(k / VW) * SL + lane) * VW + (k % VW)] = to_storage<TS>(blk[r * cols + c]);
    }
  }

  template <typename TS>
  int upload_face(const FaceBlocks& fb, int64_t n, int64_t nsl, FaceOp<TS, B>& op, std::string& err) {
    using F = FaceOp<TS, B>;
    const int nf = F::NFACE, NF = F::NF, BO = F::BO;
    std::vector<TS> hv((size_t)nsl * SL * F::KS, to_storage<TS>(0.0));
    std::vector<int32_t> hn((size_t)nsl * nf * SL, -1);
    std::vector<int8_t> hc((size_t)nsl * nf * SL, 0);
    for (int64_t u = 0; u < n; ++u) {
      const int64_t sl = u / SL;
      const int lane = (int)(u % SL);
      TS* sb = &hv[(size_t)sl * SL * F::KS];
      pack_rect<TS>(&fb.diag[(size_t)u * B * B], sb, lane, B, B);
      for (int f = 0; f < nf; ++f) {
        TS* rb = sb + (size_t)SL * (F::KP + f * (F::KR + F::KC));
        pack_rect<TS>(&fb.R[((size_t)u * nf + f) * NF * B], rb, lane, NF, B);
        pack_rect<TS>(&fb.C[((size_t)u * nf + f) * BO * NF], rb + (size_t)SL * F::KR, lane, BO, NF);
        hn[((size_t)sl * nf + f) * SL + lane] = fb.nbr[(size_t)u * nf + f];
        hc[((size_t)sl * nf + f) * SL + lane] = fb.code[(size_t)u * nf + f];
      }
    }
    TS* vals;
    int32_t* nbr;
    int8_t* code;
    int rc;
    if ((rc = upload(&vals, hv.data(), hv.size(), err))) return rc;
    if ((rc = upload(&nbr, hn.data(), hn.size(), err))) return rc;
    if ((rc = upload(&code, hc.data(), hc.size(), err))) return rc;
    op.V = FaceView<TS, B>{vals, nbr, code, nsl};
    return AGG_OK;
  }

  // B x B row-major blocks -> column-major copies in storage type TS
  template <typename TS>
  int upload_colmajor(const double* blocks, int64_t nblk, TS** out, std::string& err) {
    std::vector<TS> hv((size_t)nblk * B * B);
    for (int64_t k = 0; k < nblk; ++k)
      for (int r = 0; r < B; ++r)
        for (int c = 0; c < B; ++c)
          hv[(size_t)k * B * B + c * B + r] = to_storage<TS>(blocks[(size_t)k * B * B + r * B + c]);
    return upload(out, hv.data(), hv.size(), err);
  }

  template <typename TS>
  int upload_blocks(const std::vector<double>& blocks, int64_t n, int64_t nsl, TS** out, std::string& err) {
    constexpr int KP = Pad<TS, B>::KP;
    std::vector<TS> hv((size_t)nsl * SL * KP, to_storage<TS>(0.0));
    for (int64_t u = 0; u < n; ++u)
      pack<TS>(&blocks[(size_t)u * B * B], &hv[(size_t)(u / SL) * SL * KP], (int)(u % SL));
    return upload(out, hv.data(), hv.size(), err);
  }

  // ---------------------------------------------------------------- V-cycle
  // Launches one V-cycle from level l (rhs in lev_[l].rhs); returns the buffer
  // holding the correction.
  T* vc(int l, cudaStream_t s) {
    Lev& v = lev_[l];
    if constexpr (kRL) {
      if (cluster_ && l == lc_) return launch_cluster(s);
    }
    if (l == nlev_ - 1) {
      const int64_t g = cdiv(nc_ * 32, kCoarseNT);
      k_coarse_lower<T><<<g, kCoarseNT, 0, s>>>(Linv_, v.rhs, yc_, nc_, st_);
      k_coarse_upper<T><<<g, kCoarseNT, 0, s>>>(U_, yc_, v.xa, nc_, st_);
      return v.xa;
    }
    if constexpr (kMf) {
      if (l == 0 && mf_) return vc_level(l, mfop_, s);
    }
    if constexpr (kRL) {
      if (l == 1 && persist_) return launch_persistent(s);
    }
    if constexpr (kRowLanes) {
      if (l > 0) return vc_rowlane(l, s);
    }
    if (l == 0) return vc_level(l, fop_, s);
    return vc_level(l, SellOp<T, B>{v.A()}, s);
  }

  // Levels >= 1 and the coarsest solve in one cooperative launch; returns
  // level 1's correction (the buffer the separate kernels would end in:
  // 2 degree - 1 swaps of the ping-pong iterates).
  T* launch_persistent(cudaStream_t s) {
    if constexpr (kRL) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3((unsigned)pgrid_);
      cfg.blockDim = dim3(PNT);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, k_coarse_persistent<T, TD, kRL ? B : 4>, pc_);
    }
    return ((2 * degree_ - 1) & 1) ? lev_[1].xb : lev_[1].xa;
  }

  // Fills the persistent kernel's level table; false if the hierarchy does
  // not qualify (fewer than 3 levels, too many levels, no resident block).
  bool setup_persistent(std::string& err) {
    if constexpr (!kRL) {
      return false;
    } else {
      if (nlev_ < 3 || nlev_ - 2 >= PMAXL || degree_ > PMAXDEG) return false;
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_coarse_persistent<T, TD, kRL ? B : 4>, PNT, 0) !=
              cudaSuccess ||
          nb < 1) {
        cudaGetLastError();
        return false;
      }
      pgrid_ = num_sms_ * nb;
      if (!bar_ && dalloc(&bar_, 1, err)) return false;
      fill_table(pc_, 1);
      // test hook: barriers that wait for arrivals that never come (their
      // bounded spins then end the solve with AGG_ECUDA)
      pc_.extra = getenv("AGG_PERSIST_TEST_EXTRA") ? (unsigned)std::max(0, atoi(getenv("AGG_PERSIST_TEST_EXTRA"))) : 0u;
      return true;
    }
  }

  // Level table of the coarse-cycle kernels from level `first` on.
  void fill_table(PCoarse<T, TD>& pc, int first) {
    {
      pc = PCoarse<T, TD>{};
      pc.first = first;
      pc.nl = nlev_ - 2;
      pc.degree = degree_;
      for (int l = first; l <= pc.nl; ++l) {
        const Lev& v = lev_[l];
        PLevel<T, TD>& q = pc.lev[l];
        q.A = v.rl;
        q.Dinv = v.rl_dinv;
        q.P = v.rl_P;
        q.parent = v.parent;
        q.child_ptr = v.child_ptr;
        q.rhs = v.rhs;
        q.xa = v.xa;
        q.xb = v.xb;
        q.d = v.d;
        q.S = v.S;
        for (int k = 0; k < degree_; ++k) {
          q.c1[k] = v.c1[k];
          q.c2[k] = v.c2[k];
        }
        q.n = v.n;
      }
      const Lev& c = lev_[nlev_ - 1];
      pc.n_c_units = c.n;
      pc.child_ptr_c = c.child_ptr;
      pc.rhs_c = c.rhs;
      pc.x_c = c.xa;
      pc.Linv = Linv_;
      pc.U = U_;
      pc.yc = yc_;
      pc.nc = nc_;
      pc.bar = bar_;
      pc.st = st_;
      pc.extra = 0u;
    }
  }

  // The cluster kernel: first level lc_ (the first level whose rows fit one
  // pass of the cluster), cluster of 16 CTAs where the device schedules one,
  // else 8. False when no level qualifies below level 1 or no cluster fits.
  bool setup_cluster() {
    if constexpr (!kRL) {
      return false;
    } else {
      if (nlev_ < 2 || nlev_ - 2 >= PMAXL || degree_ > PMAXDEG) return false;
      auto kern = k_coarse_cluster<T, TD, kRL ? B : 4>;
      for (int cs : {16, 8}) {
        if (cs > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)cs);
        cfg.blockDim = dim3(CNT);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclus = 0;
        if (cudaOccupancyMaxActiveClusters(&nclus, kern, &cfg) != cudaSuccess || nclus < 1) {
          cudaGetLastError();
          continue;
        }
        const int64_t cap = (int64_t)cs * CNT;
        int lc = nlev_ - 1;
        for (int l = nlev_ - 2; l >= 1 && lev_[l].n * B <= cap; --l) lc = l;
        if (lc < 1) return false;
        lc_ = lc;
        csize_ = cs;
        fill_table(pcc_, lc_);
        return true;
      }
      return false;
    }
  }

  // Levels lc_ .. L-1 in one cluster launch; returns level lc_'s correction
  // (the coarsest's solution when lc_ is the coarsest level).
  T* launch_cluster(cudaStream_t s) {
    if constexpr (kRL) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3((unsigned)csize_);
      cfg.blockDim = dim3(CNT);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)csize_;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, k_coarse_cluster<T, TD, kRL ? B : 4>, pcc_);
    }
    if (lc_ == nlev_ - 1) return lev_[lc_].xa;
    return ((2 * degree_ - 1) & 1) ? lev_[lc_].xb : lev_[lc_].xa;
  }

  // Whether level l's first smoother step sums the finer level's
  // restriction itself (k_rl_cheb_restricted) instead of a k_segsum launch:
  // the row-lane levels run as separate kernels.
  bool fused_restrict(int l) const {
    if constexpr (!kRowLanes) return false;
    if (l < 1 || l >= nlev_ - 1) return false;
    if (l == 1 && persist_) return false;
    if (cluster_ && l >= lc_) return false;
    return true;
  }

  // Kernel launches of one V-cycle from level l: 2 degree smoother steps,
  // residual + restriction, segmented sum (unless the next level fuses it),
  // prolongation.
  int vcycle_launches(int l) const {
    if (cluster_ && l == lc_) return 1;
    if (l == nlev_ - 1) return 2;
    if (l == 1 && persist_) return 1;
    return 2 * degree_ + 3 - (fused_restrict(l + 1) ? 1 : 0) + vcycle_launches(l + 1);
  }

  // One coarse level (l >= 1) with the row-lane kernels.
  T* vc_rowlane(int l, cudaStream_t s) {
    Lev& v = lev_[l];
    T* xo = v.xa;
    T* xn = v.xb;
    const int64_t g = rl_grid<kRowLanes ? B : 1>(v.n);
    if (fused_restrict(l))
      k_rl_cheb_restricted<T, TD, B><<<g, RL_NT, 0, s>>>(v.rl, v.rl_dinv, v.child_ptr, lev_[l - 1].S, v.rhs, xo,
                                                          v.d, v.c2[0], st_);
    else
      k_rl_cheb<T, TD, B, 0><<<g, RL_NT, 0, s>>>(v.rl, v.rl_dinv, v.rhs, nullptr, xo, v.d, T(0), v.c2[0], st_);
    for (int k = 1; k < degree_; ++k) {
      k_rl_cheb<T, TD, B, 2><<<g, RL_NT, 0, s>>>(v.rl, v.rl_dinv, v.rhs, xo, xn, v.d, v.c1[k], v.c2[k], st_);
      std::swap(xo, xn);
    }
    Lev& c = lev_[l + 1];
    k_rl_resid_restrict<T, B><<<g, RL_NT, 0, s>>>(v.rl, v.rl_P, v.rhs, xo, v.S, st_);
    if (!fused_restrict(l + 1))
      k_segsum<T, B><<<cdiv(c.n * B, 256), 256, 0, s>>>(c.child_ptr, v.S, c.rhs, c.n, st_);
    T* ec = vc(l + 1, s);
    k_rl_prolong<T, B><<<g, RL_NT, 0, s>>>(v.rl_P, v.parent, ec, xo, v.n, st_);
    k_rl_cheb<T, TD, B, 1><<<g, RL_NT, 0, s>>>(v.rl, v.rl_dinv, v.rhs, xo, xn, v.d, T(0), v.c2[0], st_);
    std::swap(xo, xn);
    for (int k = 1; k < degree_; ++k) {
      k_rl_cheb<T, TD, B, 2><<<g, RL_NT, 0, s>>>(v.rl, v.rl_dinv, v.rhs, xo, xn, v.d, v.c1[k], v.c2[k], st_);
      std::swap(xo, xn);
    }
    return xo;
  }

  // Chebyshev step KIND 1 or 2 on level v with operator op
  template <int KIND, typename Op>
  void cheb_step(const Op& op, Lev& v, const T* xo, T* xn, T c1, T c2, cudaStream_t s, const CGState* st) {
    k_cheb<T, TD, B, KIND, Op><<<bgrid(0, v.nsl), NTB, 0, s>>>(op, v.Dinv, v.rhs, xo, xn, v.d, c1, c2, v.nsl, st);
  }

  // One level of the V-cycle with the level operator `op` (assembled blocks
  // or the matrix-free fine operator).
  template <typename Op>
  T* vc_level(int l, const Op& op, cudaStream_t s) {
    Lev& v = lev_[l];
    T* xo = v.xa;
    T* xn = v.xb;
    const int64_t g = bgrid(0, v.nsl);
    k_cheb<T, TD, B, 0, Op><<<g, NTB, 0, s>>>(op, v.Dinv, v.rhs, nullptr, xo, v.d, T(0), v.c2[0], v.nsl, st_);
    for (int k = 1; k < degree_; ++k) {
      cheb_step<2>(op, v, xo, xn, v.c1[k], v.c2[k], s, st_);
      std::swap(xo, xn);
    }
    Lev& c = lev_[l + 1];
    k_resid_restrict<T, B, Op><<<g, NTB, 0, s>>>(op, v.P, v.rhs, xo, v.S, st_);
    if (!fused_restrict(l + 1))
      k_segsum<T, B><<<cdiv(c.n * B, 256), 256, 0, s>>>(c.child_ptr, v.S, c.rhs, c.n, st_);
    T* ec = vc(l + 1, s);
    k_prolong<T, B, OpStreams<Op>::value><<<g, NTB, 0, s>>>(v.P, v.parent, ec, xo, v.nsl, st_);
    cheb_step<1>(op, v, xo, xn, T(0), v.c2[0], s, st_);
    std::swap(xo, xn);
    for (int k = 1; k < degree_; ++k) {
      cheb_step<2>(op, v, xo, xn, v.c1[k], v.c2[k], s, st_);
      std::swap(xo, xn);
    }
    return xo;
  }

  int64_t N0() const { return lev_[0].nvec; }
  bool use_mf0() const { return kMf && mf_; }
  int64_t g0() const { return cdiv(lev_[0].nsl * SL, NTB); }

  // z = V(r), beta, p. In the iteration body the float32 cast of r and the
  // flexible-beta product (r, z_old) come fused in k_cg_update.
  void launch_precond(cudaStream_t s, bool init) {
    const int64_t N = N0();
    if (init && !std::is_same<T, double>::value)
      k_cast<float, double><<<RED_BLOCKS, RED_NT, 0, s>>>(r_, r32_, N, st_);
    T* out = vc(0, s);
    if (init) {
      k_zdot<T, true><<<RED_BLOCKS, RED_NT, 0, s>>>(out, z_, r_, N, partials_, st_);
      k_pupd<true><<<RED_BLOCKS, RED_NT, 0, s>>>(z_, p_, N, st_);
    } else {
      k_zdot<T, false><<<RED_BLOCKS, RED_NT, 0, s>>>(out, z_, r_, N, partials_, st_);
      k_pupd<false><<<RED_BLOCKS, RED_NT, 0, s>>>(z_, p_, N, st_);
    }
  }

  void launch_init(cudaStream_t s, unsigned long long cond, int use_cond) {
    k_cg_begin<<<1, 1, 0, s>>>(st_, cond, use_cond, persist_ ? bar_ : nullptr);
    k_spmv<double, B, 1, A0Op><<<bgrid(0, lev_[0].nsl), NTB, 0, s>>>(A0f_, x_, b_, r_, nullptr, nullptr);
    k_r0<<<RED_BLOCKS, RED_NT, 0, s>>>(r_, N0(), partials_, st_);
    launch_precond(s, true);
    k_loop_ctl<<<1, 1, 0, s>>>(st_);
  }

  void launch_body(cudaStream_t s) {
    k_spmv<double, B, 2, A0Op><<<bgrid(0, lev_[0].nsl), NTB, 0, s>>>(A0f_, p_, nullptr, q_, partials_, st_);
    k_cg_update<<<RED_BLOCKS, RED_NT, 0, s>>>(x_, r_, p_, q_, std::is_same<T, double>::value ? nullptr : r32_, z_,
                                              N0(), partials_, st_);
    launch_precond(s, false);
    k_loop_ctl<<<1, 1, 0, s>>>(st_);
  }

  void launch_step_prologue(cudaStream_t s) {
    IonicParams ip{sp_.model, sp_.k, sp_.a, sp_.eps, sp_.gamma, sp_.mu1, sp_.mu2, sp_.bo};
    if (sp_.scheme == 1) {
      k_ionic_rhs_bdf2<B><<<bgrid(0, lev_[0].nsl), NTB, 0, s>>>(Me_, x_, up_, w_, wp_, mask_, b_, ip, sp_.dt, sp_.chi,
                                                              sp_.cm, sp_.iapp_value, sp_.iapp_steps, step_,
                                                              lev_[0].nsl, N0());
      return;
    }
    const double c = sp_.chi * sp_.cm / sp_.dt;
    k_ionic_rhs<B><<<bgrid(0, lev_[0].nsl), NTB, 0, s>>>(Me_, x_, w_, mask_, b_, ip, sp_.dt, sp_.chi, c,
                                                         sp_.iapp_value, sp_.iapp_steps, step_, lev_[0].nsl, N0());
  }

  // Builds [prologue] -> WHILE(body) -> [epilogue]; prologue/epilogue are
  // callables launching kernels on a capture stream.
  template <typename Pro, typename Epi>
  int build_cond_graph(Pro pro, Epi epi, cudaGraphExec_t* exec, std::string& err) {
    cudaGraph_t g;
    AGG_CK(cudaGraphCreate(&g, 0));
    graphs_.push_back(g);
    cudaGraphConditionalHandle h;
    AGG_CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraph_t gp, ge;
    AGG_CK(cudaStreamBeginCapture(cs_, cudaStreamCaptureModeThreadLocal));
    pro(cs_, (unsigned long long)h, 1);
    AGG_CK(cudaStreamEndCapture(cs_, &gp));
    graphs_.push_back(gp);
    cudaGraphNode_t n0, n1, n2;
    AGG_CK(cudaGraphAddChildGraphNode(&n0, g, nullptr, 0, gp));
    // zero-initialised parameter block (the union has no usable default constructor)
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    AGG_CK(cudaGraphAddNode(&n1, g, &n0, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    AGG_CK(cudaStreamBeginCaptureToGraph(cs_, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_body(cs_);
    AGG_CK(cudaStreamEndCapture(cs_, &body));
    AGG_CK(cudaStreamBeginCapture(cs_, cudaStreamCaptureModeThreadLocal));
    epi(cs_);
    AGG_CK(cudaStreamEndCapture(cs_, &ge));
    graphs_.push_back(ge);
    AGG_CK(cudaGraphAddChildGraphNode(&n2, g, &n1, 1, ge));
    AGG_CK(cudaGraphInstantiate(exec, g, 0));
    return AGG_OK;
  }

  template <typename F>
  int capture(F f, cudaGraphExec_t* exec, std::string& err) {
    cudaGraph_t g;
    AGG_CK(cudaStreamBeginCapture(cs_, cudaStreamCaptureModeThreadLocal));
    f(cs_);
    AGG_CK(cudaStreamEndCapture(cs_, &g));
    graphs_.push_back(g);
    AGG_CK(cudaGraphInstantiate(exec, g, 0));
    return AGG_OK;
  }

  void end_dangling_capture() {
    cudaGetLastError();
    cudaStreamCaptureStatus cst;
    if (cudaStreamIsCapturing(cs_, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
      cudaGraph_t dummy = nullptr;
      cudaStreamEndCapture(cs_, &dummy);
      if (dummy) cudaGraphDestroy(dummy);
    }
    cudaGetLastError();
  }

  void drop_solve_graphs() {
    end_dangling_capture();
    for (cudaGraphExec_t* e : {&solve_exec_, &init_exec_, &body_exec_})
      if (*e) {
        cudaGraphExecDestroy(*e);
        *e = nullptr;
      }
  }

  // The solve's graphs: set-up and iteration body (batch fallback) and the
  // conditional WHILE graph. Without the persistent kernel a refused
  // conditional node only selects the batch fallback; with it, any failure
  // is returned so that the caller can retry with the separate kernels.
  int build_solve_graphs(std::string& err) {
    int rc;
    if ((rc = capture([&](cudaStream_t c) { launch_init(c, 0, 0); }, &init_exec_, err))) return rc;
    if ((rc = capture([&](cudaStream_t c) { launch_body(c); }, &body_exec_, err))) return rc;
    std::string cerr;
    use_cond_ = build_cond_graph([&](cudaStream_t c, unsigned long long hd, int u) { launch_init(c, hd, u); },
                                 [&](cudaStream_t c) { k_noop<<<1, 1, 0, c>>>(); }, &solve_exec_, cerr) == AGG_OK;
    if (!use_cond_) {
      end_dangling_capture();
      if (persist_ || cluster_) {
        err = cerr;
        return AGG_ECUDA;
      }
    }
    return AGG_OK;
  }

  // run a prepared solve on the internal buffers; batch fallback polls `done`
  int run_solve(cudaGraphExec_t cond_exec, cudaGraphExec_t pro, cudaGraphExec_t epi, cudaStream_t s,
                std::string& err) {
    if (use_cond_) {
      AGG_CK(cudaGraphLaunch(cond_exec, s));
      return AGG_OK;
    }
    AGG_CK(cudaGraphLaunch(pro, s));
    int launched = 0;
    int batch = 4;
    for (;;) {
      for (int i = 0; i < batch; ++i) AGG_CK(cudaGraphLaunch(body_exec_, s));
      launched += batch;
      AGG_CK(cudaMemcpyAsync(st_host_, st_, sizeof(CGState), cudaMemcpyDeviceToHost, s));
      AGG_CK(cudaStreamSynchronize(s));
      if (st_host_->done || launched > st_host_->max_it + 1) break;
      batch = std::min(2 * batch, 64);
    }
    if (epi) AGG_CK(cudaGraphLaunch(epi, s));
    return AGG_OK;
  }

 public:
  ~Engine() override {
    if (cs_) cudaStreamSynchronize(cs_);
    for (auto e : {solve_exec_, init_exec_, body_exec_, step_exec_, step_pro_exec_, step_epi_exec_})
      if (e) cudaGraphExecDestroy(e);
    for (auto g : graphs_) cudaGraphDestroy(g);
    for (void* p : allocs_) cudaFree(p);
    if (st_host_) cudaFreeHost(st_host_);
    if (cs_) cudaStreamDestroy(cs_);
  }

  bool uses_conditional_graph() const override { return use_cond_; }

  int init(const HostHierarchy& h, const Mesh& m, int precision, int fine_operator, int coarse_persistent,
           int coarse_cluster, cudaStream_t s, std::string& err) override {
    (void)precision;
    mesh_ = &m;
    perm0_ = h.lev[0].perm;
    inv0_ = h.lev[0].inv;
    mass_coeff_ = h.mass_coeff;
    nlev_ = h.L;
    degree_ = 3;
    {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&num_sms_, cudaDevAttrMultiProcessorCount, dev);
    }
    lev_.assign(nlev_, Lev());
    AGG_CK(cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking));
    AGG_CK(cudaMallocHost(&st_host_, sizeof(CGState)));
    std::memset(st_host_, 0, sizeof(CGState));
    int rc;
    if ((rc = dalloc(&st_, 1, err))) return rc;
    for (int l = 0; l < nlev_; ++l) nnzb_.push_back(h.lev[l].A.nnzb());
    for (int l = 0; l < nlev_; ++l) {
      const HostLevel& hl = h.lev[l];
      Lev& v = lev_[l];
      v.n = hl.n;
      v.nsl = cdiv(hl.n, SL);
      v.nvec = v.nsl * SL * B;
      if ((rc = upload(&v.perm, hl.perm.data(), hl.perm.size(), err))) return rc;
      const bool coarsest = (l == nlev_ - 1);
      if (!coarsest) {
        // level 0 keeps its slot structure only (its operator is face-structured)
        if ((rc = upload_sell<T>(hl.A, v.nsl, &v.slice_ptr, &v.cols, &v.vals, err, l > 0))) return rc;
        if ((rc = upload_dinv(hl.Dinv, hl.n, v.nsl, &v.Dinv, err))) return rc;
        if ((rc = upload_blocks<T>(hl.P, hl.n, v.nsl, &v.P, err))) return rc;
        std::vector<int32_t> par(v.nsl * SL, 0);
        std::copy(hl.parent.begin(), hl.parent.end(), par.begin());
        if ((rc = upload(&v.parent, par.data(), par.size(), err))) return rc;
        // Chebyshev coefficients (recurrence of O10)
        const double th = 0.5 * (hl.lam_max + hl.lam_min), de = 0.5 * (hl.lam_max - hl.lam_min);
        const double sig = th / de;
        double rho = 1.0 / sig;
        v.c1.assign(degree_, T(0));
        v.c2.assign(degree_, T(0));
        v.c2[0] = T(1.0 / th);
        for (int k = 1; k < degree_; ++k) {
          const double rn = 1.0 / (2.0 * sig - rho);
          v.c1[k] = T(rn * rho);
          v.c2[k] = T(2.0 * rn / de);
          rho = rn;
        }
        if ((rc = dalloc(&v.xb, v.nvec, err))) return rc;
        if ((rc = dalloc(&v.d, v.nvec, err))) return rc;
        if ((rc = dalloc(&v.S, v.nvec, err))) return rc;
        if (kRowLanes && l > 0) {
          std::vector<int32_t> rp(hl.A.rowptr.begin(), hl.A.rowptr.end());
          int32_t *drp, *dcol;
          T* dval;
          if ((rc = upload(&drp, rp.data(), rp.size(), err))) return rc;
          if ((rc = upload(&dcol, hl.A.col.data(), hl.A.col.size(), err))) return rc;
          if ((rc = upload_colmajor<T>(hl.A.val.data(), hl.A.nnzb(), &dval, err))) return rc;
          v.rl = CsrBlocks<T>{drp, dcol, dval, hl.n};
          if ((rc = upload_colmajor<TD>(hl.Dinv.data(), hl.n, &v.rl_dinv, err))) return rc;
          if ((rc = upload_colmajor<T>(hl.P.data(), hl.n, &v.rl_P, err))) return rc;
        }
      }
      if (l > 0) {
        if ((rc = upload(&v.child_ptr, hl.child_ptr.data(), hl.child_ptr.size(), err))) return rc;
        if ((rc = dalloc(&v.rhs, v.nvec, err))) return rc;
      }
      if ((rc = dalloc(&v.xa, v.nvec, err))) return rc;
    }
    // face-structured level-0 operators: float64 (outer CG) and, for the
    // assembled smoother, the V-cycle precision
    {
      FaceBlocks fb;
      if ((rc = face_blocks_build(m, h.lev[0], fb, err))) return rc;
      int64_t nface = 0;
      for (int32_t nb : fb.nbr) nface += (nb >= 0);
      face_entries_ = (double)m.ne * B * B + (double)nface * (2.0 * fb.NF * B - (double)fb.NF * fb.NF);
      if ((rc = upload_face<double>(fb, m.ne, lev_[0].nsl, A0f_, err))) return rc;
      if constexpr (std::is_same<T, double>::value) {
        fop_ = A0f_;
      } else if (fine_operator != 1) {
        if ((rc = upload_face<T>(fb, m.ne, lev_[0].nsl, fop_, err))) return rc;
      }
      if (!lev_[0].slice_ptr) {
        if ((rc = upload_sell<double>(h.lev[0].A, lev_[0].nsl, &lev_[0].slice_ptr, &lev_[0].cols, nullptr, err, false)))
          return rc;
      }
      A0_ = SellView<double>{lev_[0].slice_ptr, lev_[0].cols, nullptr, lev_[0].nsl};
    }
    // element mass blocks in internal order for the right-hand side
    {
      std::vector<double> me((size_t)m.ne * B * B);
      for (int64_t r = 0; r < m.ne; ++r)
        std::memcpy(&me[(size_t)r * B * B], &m.Me[(size_t)h.lev[0].perm[r] * B * B], sizeof(double) * B * B);
      if ((rc = upload_blocks<double>(me, m.ne, lev_[0].nsl, &Me_, err))) return rc;
      me_int_.swap(me);
    }
    // adjoint data: volume forms and per-slot face parts in the fine operator's slot order
    if (m.adjoint_data) {
      const HostLevel& l0 = h.lev[0];
      std::vector<double> ke((size_t)m.ne * B * B);
      for (int64_t r = 0; r < m.ne; ++r)
        std::memcpy(&ke[(size_t)r * B * B], &m.Ke[(size_t)l0.perm[r] * B * B], sizeof(double) * B * B);
      if ((rc = upload_blocks<double>(ke, m.ne, lev_[0].nsl, &Ke_, err))) return rc;
      // face parts per (slice, local face), the five parts padded to whole
      // double2 chunks, in the chunk layout (see k_grad_logD); copied in
      // pieces of 1024 slices so the host needs no full-size staging copy
      using YL = AdjFaceLayout<B>;
      const int nf = 2 * FaceShape<B>::D, NF = YL::NF;
      const int64_t nsl = lev_[0].nsl;
      const size_t per_slice = (size_t)nf * YL::YS * SL;
      if ((rc = dalloc(&Y_, (size_t)nsl * per_slice, err))) return rc;
      const int sizes[5] = {NF * B, (B - NF) * NF, B * NF, NF * B, NF * NF};
      const int offs[5] = {0, YL::P1, YL::P1 + YL::P2, YL::P1 + YL::P2 + YL::P3, YL::P1 + YL::P2 + YL::P3 + YL::P4};
      const int64_t piece = 1024;
      std::vector<double> hy;
      for (int64_t s0 = 0; s0 < nsl; s0 += piece) {
        const int64_t s1 = std::min(nsl, s0 + piece);
        hy.assign((size_t)(s1 - s0) * per_slice, 0.0);
        for (int64_t r = s0 * SL; r < std::min<int64_t>(m.ne, s1 * SL); ++r) {
          const int64_t e = l0.perm[r], sl = r / SL - s0;
          const int lane = (int)(r % SL);
          for (int f = 0; f < nf; ++f) {
            const double* src = &m.Yc[((size_t)e * nf + f) * 4 * NF * B];
            double* dst = &hy[((size_t)sl * nf + f) * YL::YS * SL];
            int so = 0;
            for (int pt = 0; pt < 5; ++pt) {
              for (int k = 0; k < sizes[pt]; ++k) {
                const int kk = offs[pt] + k;
                dst[((size_t)(kk / 2) * SL + lane) * 2 + (kk % 2)] = src[so + k];
              }
              so += sizes[pt];
            }
          }
        }
        AGG_CK(cudaMemcpy(Y_ + (size_t)s0 * per_slice, hy.data(), sizeof(double) * hy.size(),
                          cudaMemcpyHostToDevice));
      }
    }
    // matrix-free fine operator for the float32 V-cycle
    if (fine_operator == 1) {
      if constexpr (kMf) {
        MatrixFreeData md;
        if ((rc = matrix_free_build(m, h.lev[0].perm, h.lev[0].inv, h.mass_coeff, md, err))) return rc;
        if (md.q != MfOpT::kDegree + 2) { err = "matrix-free operator needs quad_extra = 1"; return AGG_EUNSUPPORTED; }
        float *cell, *face;
        int32_t* nbr;
        int8_t* code;
        {
          const std::vector<float> c32(md.cell.begin(), md.cell.end()), f32(md.face.begin(), md.face.end());
          if ((rc = upload(&cell, c32.data(), c32.size(), err))) return rc;
          if ((rc = upload(&face, f32.data(), f32.size(), err))) return rc;
        }
        if ((rc = upload(&nbr, md.nbr.data(), md.nbr.size(), err))) return rc;
        if ((rc = upload(&code, md.code.data(), md.code.size(), err))) return rc;
        mfop_.V = MfView{cell, face, nbr, code, lev_[0].nsl};
        Tables1D t1 = make_tables(m.p, md.q);
        std::memset(&mfop_.T, 0, sizeof(mfop_.T));
        for (int a = 0; a <= m.p; ++a) {
          for (int kq = 0; kq < md.q; ++kq) {
            double v[8], dv[8];
            lagrange_eval(t1.gll.data(), m.p + 1, t1.gx[kq], v, dv);
            mfop_.T.L[a][kq] = (float)v[a];
            mfop_.T.D[a][kq] = (float)dv[a];
          }
          for (int sd = 0; sd < 2; ++sd) {
            double v[8], dv[8];
            lagrange_eval(t1.gll.data(), m.p + 1, (double)sd, v, dv);
            mfop_.T.Dend[sd][a] = (float)dv[a];
          }
        }
        mf_bytes_ = (int64_t)(md.cell.size() * 4 + md.face.size() * 4 + md.nbr.size() * 4 + md.code.size());
        mf_ = true;
      } else {
        err = "the matrix-free fine operator needs quadrilaterals or hexahedra of p <= 3 and a float32 V-cycle";
        return AGG_EUNSUPPORTED;
      }
    }
    // coarsest: inverse Cholesky factor and its transpose
    nc_ = h.nc;
    {
      std::vector<double> Ut((size_t)nc_ * nc_);
      for (int64_t i = 0; i < nc_; ++i)
        for (int64_t j = 0; j < nc_; ++j) Ut[(size_t)j * nc_ + i] = h.Linv[(size_t)i * nc_ + j];
      if ((rc = upload(&Linv_, h.Linv.data(), h.Linv.size(), err))) return rc;
      if ((rc = upload(&U_, Ut.data(), Ut.size(), err))) return rc;
      if ((rc = dalloc(&yc_, nc_, err))) return rc;
    }
    const int64_t N = N0();
    for (double** pp : {&b_, &x_, &r_, &p_, &q_, &z_})
      if ((rc = dalloc(pp, N, err))) return rc;
    if (!std::is_same<T, double>::value)
      if ((rc = dalloc(&r32_, N, err))) return rc;
    const int64_t nparts = std::max<int64_t>(2 * RED_BLOCKS, 2 * g0() + 64);
    if ((rc = dalloc(&partials_, nparts, err))) return rc;
    lev_[0].rhs = std::is_same<T, double>::value ? reinterpret_cast<T*>(r_) : reinterpret_cast<T*>(r32_);
    AGG_CK(cudaDeviceSynchronize());
    // graphs: conditional WHILE solve, with the batch fallback prepared as
    // well; if the runtime refuses the cooperative launch of the coarse-level
    // kernel inside a graph, the separate coarse kernels are captured instead
    persist_ = coarse_persistent && setup_persistent(err);
    cluster_ = !persist_ && coarse_cluster && setup_cluster();
    for (;;) {
      rc = build_solve_graphs(err);
      if (rc == AGG_OK || (!persist_ && !cluster_)) break;
      drop_solve_graphs();
      if (persist_) persist_ = false;
      else cluster_ = false;
    }
    if (rc) return rc;
    if (getenv("AGG_NO_COND_GRAPH")) use_cond_ = false;
    (void)s;
    return AGG_OK;
  }

  int pcg_solve(const double* b_user, double* x_user, const SolveOpts& o, SolveResult& res, cudaStream_t s,
                std::string& err) override {
    const Lev& v0 = lev_[0];
    const int64_t ne = v0.n;
    const int64_t g = cdiv(ne * B, 256);
    k_gather_units<double, double><<<g, 256, 0, s>>>(b_user, b_, v0.perm, ne, B);
    k_gather_units<double, double><<<g, 256, 0, s>>>(x_user, x_, v0.perm, ne, B);
    k_set_opts<<<1, 1, 0, s>>>(st_, o.rtol, o.atol, o.max_it, o.flexible);
    int rc = run_solve(solve_exec_, init_exec_, nullptr, s, err);
    if (rc) return rc;
    k_scatter_units<double, double><<<g, 256, 0, s>>>(x_, x_user, v0.perm, ne, B);
    AGG_CK(cudaMemcpyAsync(st_host_, st_, sizeof(CGState), cudaMemcpyDeviceToHost, s));
    AGG_CK(cudaStreamSynchronize(s));
    AGG_CK(cudaGetLastError());
    res.iterations = st_host_->iter;
    res.r0 = st_host_->r0;
    res.rn = std::sqrt(st_host_->rr);
    res.status = st_host_->status;
    if (res.status == AGG_ECUDA) {
      err = "a grid barrier of the coarse-level kernel timed out; the solve was stopped";
      return AGG_ECUDA;
    }
    return AGG_OK;
  }

  int apply_level(int l, const double* x_user, double* y_user, cudaStream_t s, std::string& err) override {
    if (l == -1) {
      // the V-cycle's level-0 operator in its own precision (matrix-free if selected)
      Lev& v = lev_[0];
      const int64_t g = cdiv(v.n * B, 256);
      k_gather_units<T, double><<<g, 256, 0, s>>>(x_user, v.xa, v.perm, v.n, B);
      if (use_mf0())
        k_op_apply<T, B, MfOpT><<<bgrid(0, v.nsl), NTB, 0, s>>>(mfop_, v.xa, v.xb);
      else
        k_op_apply<T, B, L0Op><<<bgrid(0, v.nsl), NTB, 0, s>>>(fop_, v.xa, v.xb);
      k_scatter_units<double, T><<<g, 256, 0, s>>>(v.xb, y_user, v.perm, v.n, B);
      AGG_CK(cudaGetLastError());
      return AGG_OK;
    }
    if (l == -2) {
      // the float64 matrix-free level-0 operator
      int rc;
      if ((rc = build_mf64(err))) return rc;
      if constexpr (kMf64) {
        Lev& v = lev_[0];
        const int64_t g = cdiv(v.n * B, 256);
        k_gather_units<double, double><<<g, 256, 0, s>>>(x_user, p_, v.perm, v.n, B);
        k_op_apply<double, B, Mf64T><<<bgrid(0, v.nsl), NTB, 0, s>>>(mf64_, p_, q_);
        k_scatter_units<double, double><<<g, 256, 0, s>>>(q_, y_user, v.perm, v.n, B);
        AGG_CK(cudaGetLastError());
      }
      return AGG_OK;
    }
    if (l < 0 || l >= nlev_) { err = "level out of range"; return AGG_EINVAL; }
    Lev& v = lev_[l];
    const int64_t g = cdiv(v.n * B, 256);
    if (l == 0) {
      k_gather_units<double, double><<<g, 256, 0, s>>>(x_user, p_, v.perm, v.n, B);
      k_spmv<double, B, 0, A0Op><<<bgrid(0, v.nsl), NTB, 0, s>>>(A0f_, p_, nullptr, q_, nullptr, nullptr);
      k_scatter_units<double, double><<<g, 256, 0, s>>>(q_, y_user, v.perm, v.n, B);
    } else {
      if (l == nlev_ - 1) { err = "the coarsest level is applied through its Cholesky factor only"; return AGG_EUNSUPPORTED; }
      k_gather_units<T, double><<<g, 256, 0, s>>>(x_user, v.xa, v.perm, v.n, B);
      k_spmv<T, B, 0, SellOp<T, B>><<<bgrid(0, v.nsl), NTB, 0, s>>>(SellOp<T, B>{v.A()}, v.xa, nullptr, v.xb, nullptr, nullptr);
      k_scatter_units<double, T><<<g, 256, 0, s>>>(v.xb, y_user, v.perm, v.n, B);
    }
    AGG_CK(cudaGetLastError());
    return AGG_OK;
  }

  int vcycle_apply(const double* r_user, double* z_user, cudaStream_t s, std::string& err) override {
    Lev& v = lev_[0];
    const int64_t g = cdiv(v.n * B, 256);
    k_cg_reset<<<1, 1, 0, s>>>(st_, persist_ ? bar_ : nullptr);
    k_gather_units<double, double><<<g, 256, 0, s>>>(r_user, r_, v.perm, v.n, B);
    if (!std::is_same<T, double>::value)
      k_cast<float, double><<<RED_BLOCKS, RED_NT, 0, s>>>(r_, r32_, N0(), st_);
    T* out = vc(0, s);
    k_scatter_units<double, T><<<g, 256, 0, s>>>(out, z_user, v.perm, v.n, B);
    AGG_CK(cudaGetLastError());
    return AGG_OK;
  }

  int64_t level_scratch_entries(int l) const override {
    if (l < 0 || l >= nlev_) return -1;
    return lev_[l].nvec;
  }

  int apply_level_scratch(int l, const double* x_user, double* y_user, void* s_in, void* s_out, cudaStream_t s,
                          std::string& err) override {
    if (l < 0 || l >= nlev_ - 1) { err = "level out of range (the coarsest level has no stored operator)"; return AGG_EINVAL; }
    Lev& v = lev_[l];
    const int64_t g = cdiv(v.n * B, 256);
    if (l == 0) {
      double* xi = static_cast<double*>(s_in);
      double* yi = static_cast<double*>(s_out);
      k_gather_units<double, double><<<g, 256, 0, s>>>(x_user, xi, v.perm, v.n, B);
      k_spmv<double, B, 0, A0Op><<<bgrid(0, v.nsl), NTB, 0, s>>>(A0f_, xi, nullptr, yi, nullptr, nullptr);
      k_scatter_units<double, double><<<g, 256, 0, s>>>(yi, y_user, v.perm, v.n, B);
    } else {
      T* xi = static_cast<T*>(s_in);
      T* yi = static_cast<T*>(s_out);
      k_gather_units<T, double><<<g, 256, 0, s>>>(x_user, xi, v.perm, v.n, B);
      k_spmv<T, B, 0, SellOp<T, B>><<<bgrid(0, v.nsl), NTB, 0, s>>>(SellOp<T, B>{v.A()}, xi, nullptr, yi, nullptr, nullptr);
      k_scatter_units<double, T><<<g, 256, 0, s>>>(yi, y_user, v.perm, v.n, B);
    }
    AGG_CK(cudaGetLastError());
    return AGG_OK;
  }

  int sim_create(const SimParams& p, const double* mask_user, cudaStream_t s, std::string& err) override {
    if (sim_) { err = "a simulation already uses this hierarchy"; return AGG_EINVAL; }
    sp_ = p;
    int rc;
    const int64_t N = N0();
    if (!w_) {
      if ((rc = dalloc(&w_, kMaxGates * N, err))) return rc;     // gate-major, stride N
      if ((rc = dalloc(&mask_, N, err))) return rc;
      if ((rc = dalloc(&step_, 1, err))) return rc;
      if ((rc = dalloc(&iters_, cap_, err))) return rc;
      if ((rc = dalloc(&slot_, 1, err))) return rc;
      if ((rc = dalloc(&sim_status_, 1, err))) return rc;
    }
    const Lev& v0 = lev_[0];
    if (p.scheme == 1 && !up_) {
      if ((rc = dalloc(&up_, N, err))) return rc;
      if ((rc = dalloc(&wp_, kMaxGates * N, err))) return rc;
      std::vector<double> minv(me_int_.size());
      if (!spd_inverse_blocks(me_int_.data(), v0.n, B, minv.data())) { err = "element mass block not SPD"; return AGG_ENOTSPD; }
      if ((rc = upload_blocks<double>(minv, v0.n, v0.nsl, &Minv_, err))) return rc;
    }
    hist_valid_ = false;
    if (mask_user)
      k_gather_units<double, double><<<cdiv(v0.n * B, 256), 256, 0, s>>>(mask_user, mask_, v0.perm, v0.n, B);
    AGG_CK(cudaMemsetAsync(step_, 0, sizeof(int64_t), s));
    AGG_CK(cudaStreamSynchronize(s));
    if (step_exec_) { cudaGraphExecDestroy(step_exec_); step_exec_ = nullptr; }
    if (step_pro_exec_) { cudaGraphExecDestroy(step_pro_exec_); step_pro_exec_ = nullptr; }
    if (step_epi_exec_) { cudaGraphExecDestroy(step_epi_exec_); step_epi_exec_ = nullptr; }
    auto pro = [&](cudaStream_t c, unsigned long long hd, int u) {
      launch_step_prologue(c);
      launch_init(c, hd, u);
    };
    auto epi = [&](cudaStream_t c) { k_step_end<<<1, 1, 0, c>>>(st_, step_, iters_, slot_, cap_, sim_status_); };
    if (use_cond_) {
      if ((rc = build_cond_graph(pro, epi, &step_exec_, err))) return rc;
    } else {
      if ((rc = capture([&](cudaStream_t c) { pro(c, 0, 0); }, &step_pro_exec_, err))) return rc;
      if ((rc = capture(epi, &step_epi_exec_, err))) return rc;
    }
    sim_ = true;
    return AGG_OK;
  }

  int sim_step(int n_steps, double* u_user, double* w_user, int* iters_host, int64_t& clock, cudaStream_t s,
               std::string& err) override {
    if (!sim_) { err = "no simulation"; return AGG_EINVAL; }
    const Lev& v0 = lev_[0];
    const int64_t g = cdiv(v0.n * B, 256);
    k_gather_units<double, double><<<g, 256, 0, s>>>(u_user, x_, v0.perm, v0.n, B);
    const int ng = ionic_gates(sp_.model);
    const int64_t nu = v0.n * B;                  // caller's DoFs per gate
    for (int k = 0; k < ng; ++k)
      k_gather_units<double, double><<<g, 256, 0, s>>>(w_user + k * nu, w_ + k * N0(), v0.perm, v0.n, B);
    AGG_CK(cudaMemcpyAsync(step_, &clock, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    AGG_CK(cudaMemsetAsync(sim_status_, 0, sizeof(int), s));
    if (sp_.scheme == 1 && !hist_valid_) {
      // second-order start of the BDF2 history from the current state
      IonicParams ip{sp_.model, sp_.k, sp_.a, sp_.eps, sp_.gamma, sp_.mu1, sp_.mu2, sp_.bo};
      const double c = 1.5 * sp_.chi * sp_.cm / sp_.dt;
      const double ia = (clock < sp_.iapp_steps) ? sp_.iapp_value : 0.0;
      k_spmv<double, B, 0, A0Op><<<bgrid(0, v0.nsl), NTB, 0, s>>>(A0f_, x_, nullptr, q_, nullptr, nullptr);
      k_bdf2_start<B><<<bgrid(0, v0.nsl), NTB, 0, s>>>(Minv_, q_, x_, w_, mask_, up_, wp_, ip, sp_.dt, sp_.chi, sp_.cm,
                                                       c, ia, v0.nsl, N0());
      hist_valid_ = true;
    }
    k_set_opts<<<1, 1, 0, s>>>(st_, sp_.pcg.rtol, sp_.pcg.atol, sp_.pcg.max_it, sp_.pcg.flexible);
    int done = 0;
    int status = 0;
    std::vector<int> its;
    while (done < n_steps) {
      const int chunk = std::min(cap_, n_steps - done);
      AGG_CK(cudaMemsetAsync(slot_, 0, sizeof(int), s));
      for (int i = 0; i < chunk; ++i) {
        int rc = run_solve(step_exec_, step_pro_exec_, step_epi_exec_, s, err);
        if (rc) return rc;
      }
      if (iters_host) {
        its.resize(chunk);
        AGG_CK(cudaMemcpyAsync(its.data(), iters_, sizeof(int) * chunk, cudaMemcpyDeviceToHost, s));
        AGG_CK(cudaStreamSynchronize(s));
        std::copy(its.begin(), its.end(), iters_host + done);
      }
      done += chunk;
    }
    k_scatter_units<double, double><<<g, 256, 0, s>>>(x_, u_user, v0.perm, v0.n, B);
    for (int k = 0; k < ng; ++k)
      k_scatter_units<double, double><<<g, 256, 0, s>>>(w_ + k * N0(), w_user + k * nu, v0.perm, v0.n, B);
    AGG_CK(cudaMemcpyAsync(&status, sim_status_, sizeof(int), cudaMemcpyDeviceToHost, s));
    AGG_CK(cudaStreamSynchronize(s));
    AGG_CK(cudaGetLastError());
    clock += n_steps;
    return status;
  }

  int kernel_loop(int id, int reps, cudaStream_t s, std::string& err) override {
    if (id == 5) {
      int rc;
      if ((rc = build_mf64(err))) return rc;
      if constexpr (kMf64) {
        for (int i = 0; i < reps; ++i)
          k_spmv<double, B, 0, Mf64T><<<bgrid(0, lev_[0].nsl), NTB, 0, s>>>(mf64_, p_, nullptr, q_, nullptr, nullptr);
        AGG_CK(cudaGetLastError());
      }
      return AGG_OK;
    }
    if (id >= 1 && id <= 3 && nlev_ < 2) { err = "kernels 1-3 need a smoothed level 0 (n_levels >= 2)"; return AGG_EUNSUPPORTED; }
    Lev& v = lev_[0];
    const int64_t n = v.nsl;
    for (int i = 0; i < reps; ++i) {
      switch (id) {
        case 0:
          k_spmv<double, B, 0, A0Op><<<bgrid(0, n), NTB, 0, s>>>(A0f_, p_, nullptr, q_, nullptr, nullptr);
          break;
        case 1:
          if (use_mf0())
            cheb_step<2>(mfop_, v, v.xa, v.xb, v.c1[1], v.c2[1], s, nullptr);
          else
            k_cheb<T, TD, B, 2, L0Op><<<bgrid(0, n), NTB, 0, s>>>(fop_, v.Dinv, v.rhs, v.xa, v.xb, v.d, v.c1[1],
                                                                  v.c2[1], v.nsl, nullptr);
          break;
        case 2:
          if (use_mf0())
            k_resid_restrict<T, B, MfOpT><<<bgrid(0, n), NTB, 0, s>>>(mfop_, v.P, v.rhs, v.xa, v.S, nullptr);
          else
            k_resid_restrict<T, B, L0Op><<<bgrid(0, n), NTB, 0, s>>>(fop_, v.P, v.rhs, v.xa, v.S, nullptr);
          break;
        case 3:
          k_prolong<T, B><<<bgrid(k_prolong<T, B>, n), NTB, 0, s>>>(v.P, v.parent, lev_[1].xa, v.xb, v.nsl, nullptr);
          break;
        default: err = "unknown kernel id"; return AGG_EINVAL;
      }
    }
    AGG_CK(cudaGetLastError());
    return AGG_OK;
  }

  void launch_counts(int& per_vcycle, int& per_iteration, int& per_setup, int& persistent, int& cluster_level,
                     int& cluster_ctas) const override {
    cluster_level = cluster_ ? lc_ : -1;
    cluster_ctas = cluster_ ? csize_ : 0;
    per_vcycle = vcycle_launches(0);
    per_iteration = 5 + per_vcycle;   // SpMV + (p, q), CG update, V-cycle, (r, z), p update, loop control
    per_setup = 6 + (std::is_same<T, double>::value ? 0 : 1) + per_vcycle;   // begin, residual, ||r0||, [cast], V-cycle, (r, z), p, loop control
    persistent = persist_ ? 1 : 0;
  }

  int kernel_cost(int id, double& bytes, double& flops) const override {
    if (id >= 1 && id <= 4 && nlev_ < 2) return AGG_EUNSUPPORTED;
    const double n0 = (double)lev_[0].n, N = n0 * B, bb = (double)B * B;
    const double sT = sizeof(T), sD = sizeof(TD);
    const double bd = (B <= 32) ? (double)SymPad<TD, B>::NP : bb;   // stored smoother entries
    // face-structured operator: its stored entries and, per face slot, a
    // neighbour id and a face code
    const double fidx = n0 * 2 * FaceShape<B>::D * 5.0;
    const double fe = face_entries_;
    switch (id) {
      case 0: bytes = fe * 8 + fidx + 2 * N * 8; flops = 2 * fe; break;
      case 1:
        bytes = (use_mf0() ? (double)mf_bytes_ : fe * sT + fidx) + n0 * bd * sD + 5 * N * sT;
        flops = 2 * fe + 2 * n0 * bb + 4 * N;
        break;
      case 2:
        bytes = (use_mf0() ? (double)mf_bytes_ : fe * sT + fidx) + n0 * bb * sT + 3 * N * sT;
        flops = 2 * fe + 2 * n0 * bb + N;
        break;
      case 3: bytes = n0 * bb * sT + 2 * N * sT + (double)lev_[1].n * B * sT + n0 * 4; flops = 2 * n0 * bb + N; break;
      case 4: iteration_cost(bytes, flops); break;
      case 5:
        if (!mf64_ready_) return AGG_EUNSUPPORTED;
        bytes = (double)mf64_bytes_ + 2 * N * 8;
        flops = 2 * fe;
        break;
      default: return AGG_EINVAL;
    }
    return AGG_OK;
  }

  // Algorithmic bytes and flops of one iteration of the solve body: the
  // float64 SpMV, the CG update, one V-cycle over every level, the z and p
  // updates. Each launch reads its operator, block and vector entries once
  // and writes each output once; flops count two per stored matrix entry
  // used (the matrix-free level-0 operator as its assembled counterpart).
  void iteration_cost(double& bytes, double& flops) const {
    const double bb = (double)B * B, sT = sizeof(T), sD = sizeof(TD);
    const double n0 = (double)lev_[0].n, N = n0 * B, fe = face_entries_;
    const double fidx = n0 * 2 * FaceShape<B>::D * 5.0;
    const double deg = degree_;
    // outer CG: SpMV (p in, q out), update (x, r, p, q in; x, r out; the
    // float32 copy of r and the flexible (r, z_old) read in the reduced-
    // precision forms), z = V(r) with (r, z), p = z + beta p
    const bool lowp = !std::is_same<T, double>::value;
    bytes = fe * 8 + fidx + 2 * N * 8;
    bytes += 6 * N * 8 + (lowp ? N * 4 + N * 8 : 0.0);
    bytes += N * sT + 2 * N * 8 + 3 * N * 8;
    flops = 2 * fe + 12 * N;
    for (int l = 0; l < nlev_; ++l) {
      const double nl = (double)lev_[l].n, Nl = nl * B;
      if (l == nlev_ - 1) {                                 // two dense triangular products
        const double nc = (double)nc_;
        bytes += 2 * nc * nc * 8 + 2 * nc * sT + 2 * nc * 8;
        flops += 4 * nc * nc;
        break;
      }
      const double Nc = (double)lev_[l + 1].n * B;
      double op, opf, dinv;
      if (l == 0) {
        op = use_mf0() ? (double)mf_bytes_ : fe * sT + fidx;
        opf = 2 * fe;
        dinv = nl * ((B <= 32) ? (double)SymPad<TD, B>::NP : bb) * sD;
      } else {
        const double nz = (double)nnzb_[l];
        op = nz * bb * sT + nz * 4 + (nl + 1) * 4;
        opf = 2 * nz * bb;
        dinv = nl * bb * sD;                                // full blocks on levels >= 1
      }
      const double P = nl * bb * sT;
      // 2 deg smoother steps (2 deg - 1 with an operator product: the first
      // step from x = 0 has none), residual + restriction, segmented sum,
      // prolongation
      bytes += 2 * deg * op + 2 * deg * dinv + 2 * P;
      bytes += (3 + 2 * (deg - 1) * 5 + 4) * Nl * sT;      // smoother vectors
      bytes += 3 * Nl * sT + (Nl + Nc) * sT + ((double)lev_[l + 1].n + 1) * 8 + (Nc + 2 * Nl) * sT + nl * 4;
      flops += 2 * deg * opf + 2 * deg * 2 * nl * bb + 2 * 2 * nl * bb + 10 * deg * Nl;
    }
  }

  int adjoint_step(const double* u_n, const double* w_n, const double* u_np1, double* ubar, double* wbar,
                   double* grad, SolveResult& res, cudaStream_t s, std::string& err) override {
    if (!sim_) { err = "no simulation"; return AGG_EINVAL; }
    if (!Ke_ || !Y_) { err = "the mesh was created without adjoint data (agg_mesh_desc.adjoint_data)"; return AGG_EINVAL; }
    if (sp_.scheme != 0) { err = "the adjoint step is built for the backward-Euler scheme"; return AGG_EUNSUPPORTED; }
    if (ionic_gates(sp_.model) != 1) { err = "the adjoint step is built for one-gate ionic models"; return AGG_EUNSUPPORTED; }
    int rc;
    const int64_t N = N0();
    if (!ua_) {
      for (double** pp : {&ua_, &wa_, &ub_, &wb_})
        if ((rc = dalloc(pp, N, err))) return rc;
    }
    const Lev& v0 = lev_[0];
    const int64_t g = cdiv(v0.n * B, 256);
    // lambda = K^{-1} ubar by the same MG-PCG, from a zero guess
    k_gather_units<double, double><<<g, 256, 0, s>>>(ubar, b_, v0.perm, v0.n, B);
    AGG_CK(cudaMemsetAsync(x_, 0, sizeof(double) * N, s));
    k_set_opts<<<1, 1, 0, s>>>(st_, sp_.pcg.rtol, sp_.pcg.atol, sp_.pcg.max_it, sp_.pcg.flexible);
    if ((rc = run_solve(solve_exec_, init_exec_, nullptr, s, err))) return rc;
    k_gather_units<double, double><<<g, 256, 0, s>>>(u_n, ua_, v0.perm, v0.n, B);
    k_gather_units<double, double><<<g, 256, 0, s>>>(w_n, wa_, v0.perm, v0.n, B);
    k_gather_units<double, double><<<g, 256, 0, s>>>(u_np1, ub_, v0.perm, v0.n, B);
    k_gather_units<double, double><<<g, 256, 0, s>>>(wbar, wb_, v0.perm, v0.n, B);
    IonicParams ip{sp_.model, sp_.k, sp_.a, sp_.eps, sp_.gamma, sp_.mu1, sp_.mu2, sp_.bo};
    const double c = sp_.chi * sp_.cm / sp_.dt;
    k_adj_pointwise<B><<<bgrid(k_adj_pointwise<B>, v0.nsl), NTB, 0, s>>>(Me_, x_, ua_, wa_, b_, wb_, ip, sp_.dt, sp_.chi, c, v0.nsl);
    k_grad_logD<B><<<bgrid(0, v0.nsl), NTB, 0, s>>>(A0f_.V, Ke_, Y_, x_, ub_, v0.perm, grad, v0.n);
    k_scatter_units<double, double><<<g, 256, 0, s>>>(b_, ubar, v0.perm, v0.n, B);
    k_scatter_units<double, double><<<g, 256, 0, s>>>(wb_, wbar, v0.perm, v0.n, B);
    AGG_CK(cudaMemcpyAsync(st_host_, st_, sizeof(CGState), cudaMemcpyDeviceToHost, s));
    AGG_CK(cudaStreamSynchronize(s));
    AGG_CK(cudaGetLastError());
    res.iterations = st_host_->iter;
    res.r0 = st_host_->r0;
    res.rn = std::sqrt(st_host_->rr);
    res.status = st_host_->status;
    return AGG_OK;
  }

  void sim_invalidate_history() override { hist_valid_ = false; }

  int sim_destroy() override {
    sim_ = false;
    return AGG_OK;
  }
};

}  // namespace aggmg
