// Tile-level symbolic analysis of the local factorisations. K_rr^(k) is banded
// in the library's r_V order (lexicographic in the control index, see
// model.cpp), so most 64 x 64 tiles of its Cholesky factor stay zero. The
// pattern of nonzero tiles of K_rr is found once from an assembled matrix (it
// does not depend on the reluctivities), the fill of the factor follows from
// the block elimination on the host, and from it:
//   - the work lists of the blocked factorisation (panel solves and trailing
//     updates of nonzero tiles only, in the same step schedule as the dense
//     factorisation: two panels per FP32 trailing update unless the S_rIrI
//     snapshot falls between them, one panel in FP64),
//   - the nonzero tiles of every block row and block column of the factor for
//     the triangular sweeps,
//   - per-tile flags for the multi-column solves,
//   - the nonzero tiles of every block row of K_rr for the refinement residual.
// Skipping a zero tile is exact: its entries are zero in K_rr and no update
// reaches them.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace ieti {

namespace {

// flags[fo_k + I + nblk J] = 1 when an entry of rows 64 I.., columns 64 J.. of
// K_rr^(k) is nonzero (one warp per tile)
__global__ void k_tile_flags(const SubDev* sd, const int64_t* fo, const double* K64, unsigned char* flags) {
  const int k = blockIdx.y;
  const SubDev s = sd[k];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t nt = (int64_t)s.nblk * s.nblk;
  for (int64_t t = (int64_t)blockIdx.x * 8 + warp; t < nt; t += (int64_t)gridDim.x * 8) {
    const int I = (int)(t % s.nblk), J = (int)(t / s.nblk);
    const double* base = K64 + s.A + (int64_t)I * NB + (int64_t)s.n * J * NB;
    bool nz = false;
    for (int c = 0; c < NB; ++c) {
      const double2 v = reinterpret_cast<const double2*>(base + (int64_t)s.n * c)[lane];
      nz |= (v.x != 0.0) || (v.y != 0.0);
    }
    nz = __any_sync(0xffffffffu, nz);
    if (lane == 0) flags[fo[k] + t] = nz ? 1 : 0;
  }
}

}  // namespace

ieti_status build_ktiles(Ctx* c, cudaStream_t st) {
  const int nsub = c->nsub;
  c->tile_off.assign(nsub + 1, 0);
  c->blk_base.assign(nsub + 1, 0);
  for (int k = 0; k < nsub; ++k) {
    const int m = c->sd_host[k].nblk;
    c->tile_off[k + 1] = c->tile_off[k] + (int64_t)m * m;
    c->blk_base[k + 1] = c->blk_base[k] + m;
  }
  const int64_t nf = c->tile_off[nsub];
  int64_t* d_fo = nullptr;
  unsigned char* d_flags = nullptr;
  IETI_CUDA_TRY(c, cudaMalloc(&d_fo, sizeof(int64_t) * std::max(nsub, 1)));
  IETI_CUDA_TRY(c, cudaMalloc(&d_flags, std::max<int64_t>(nf, 1)));
  IETI_CUDA_TRY(c, cudaMemcpyAsync(d_fo, c->tile_off.data(), sizeof(int64_t) * nsub, cudaMemcpyHostToDevice, st));
  k_tile_flags<<<dim3(256, nsub), 256, 0, st>>>(c->d_sd, d_fo, c->K64, d_flags);
  IETI_LAUNCH_CHECK(c);
  c->kflags.assign(nf, 0);
  IETI_CUDA_TRY(c, cudaMemcpyAsync(c->kflags.data(), d_flags, nf, cudaMemcpyDeviceToHost, st));
  IETI_CUDA_TRY(c, cudaStreamSynchronize(st));
  cudaFree(d_fo);
  cudaFree(d_flags);
  // block row I of K_rr lists the J with tile (J, I) nonzero: row r of block I
  // reads column r (K_rr is symmetric), i.e. entries of rows 64 J.. of column block I
  const int nb = c->blk_base[nsub];
  std::vector<int64_t> trow(nb + 1, 0);
  std::vector<int32_t> tcol;
  for (int k = 0; k < nsub; ++k) {
    const int m = c->sd_host[k].nblk;
    for (int I = 0; I < m; ++I) {
      trow[c->blk_base[k] + I] = (int64_t)tcol.size();
      for (int J = 0; J < m; ++J)
        if (c->kflags[c->tile_off[k] + J + (int64_t)m * I]) tcol.push_back(J);
    }
  }
  trow[nb] = (int64_t)tcol.size();
  if (tcol.empty()) tcol.push_back(0);
  std::vector<int4> kt;
  for (int k = 0; k < nsub; ++k) {
    const int m = c->sd_host[k].nblk;
    for (int J = 0; J < m; ++J)
      for (int I = 0; I < m; ++I)
        // the lower tiles: the Kronecker assembly writes each with its mirror
        if (I >= J && c->kflags[c->tile_off[k] + I + (int64_t)m * J]) kt.push_back(make_int4(k, I, J, 0));
  }
  c->n_ktiles = (int)kt.size();
  if (kt.empty()) kt.push_back(make_int4(0, 0, 0, 0));
  ieti_status r;
  if ((r = dev_upload(c, &c->d_ktile_row, trow)) != IETI_OK) return r;
  if ((r = dev_upload(c, &c->d_ktile_col, tcol)) != IETI_OK) return r;
  if ((r = dev_upload(c, &c->d_ktile_base, c->blk_base)) != IETI_OK) return r;
  if ((r = dev_upload(c, &c->d_ktile_list, kt)) != IETI_OK) return r;
  c->ktile_ready = true;
  return IETI_OK;
}

ieti_status build_symbolic(Ctx* c, cudaStream_t st) {
  ieti_status r;
  if (!c->ktile_ready && (r = build_ktiles(c, st)) != IETI_OK) return r;
  const int nsub = c->nsub;
  // ---- fill of the factor: lower tiles, block elimination
  std::vector<unsigned char>& F = c->lflags;
  F.assign(c->tile_off[nsub], 0);
  for (int k = 0; k < nsub; ++k) {
    const int m = c->sd_host[k].nblk;
    unsigned char* T = F.data() + c->tile_off[k];   // T[i + m j], i >= j
    const unsigned char* Kf = c->kflags.data() + c->tile_off[k];
    for (int j = 0; j < m; ++j)
      for (int i = j; i < m; ++i) T[i + (int64_t)m * j] = (i == j) || Kf[i + (int64_t)m * j] || Kf[j + (int64_t)m * i];
    std::vector<int> R;
    for (int j = 0; j < m; ++j) {
      R.clear();
      for (int i = j + 1; i < m; ++i)
        if (T[i + (int64_t)m * j]) R.push_back(i);
      for (size_t a = 0; a < R.size(); ++a)
        for (size_t b2 = 0; b2 <= a; ++b2) T[R[a] + (int64_t)m * R[b2]] = 1;
    }
  }
  auto L = [&](int k, int i, int j) -> bool {
    const int m = c->sd_host[k].nblk;
    return i < m && j < m && i >= j && F[c->tile_off[k] + i + (int64_t)m * j];
  };
  // ---- factorisation work lists, FP32 (pair tiles, two panels) and FP64 (single tiles)
  const int M = c->max_nblk;
  auto snap_at = [&](int b) {
    for (auto& s : c->sd_host)
      if (s.nVp == b * NB && s.nI > 0) return true;
    return false;
  };
  for (int prec = 0; prec < 2; ++prec) {   // 0: FP64, 1: FP32
    FactorPlan& P = c->fplan[prec];
    P.steps.clear();
    std::vector<int4> items;
    std::vector<int2> trsm;
    auto add_trsm = [&](int b, int64_t* off, int* cnt) {
      *off = (int64_t)trsm.size();
      for (int k = 0; k < nsub; ++k)
        for (int rr = b + 1; rr < c->sd_host[k].nblk; ++rr)
          if (L(k, rr, b)) trsm.push_back(make_int2(k, rr));
      *cnt = (int)((int64_t)trsm.size() - *off);
    };
    for (int b = 0; b < M;) {
      FactorStep S{};
      S.b = b;
      S.snap = snap_at(b);
      S.kb = (prec == 1 && !c->syrk_tc && b + 2 < M && !snap_at(b + 1)) ? 2 : 1;
      add_trsm(b, &S.trsm_off[0], &S.trsm_cnt[0]);
      if (S.kb == 2) {
        // block column b+1 takes panel b's update: pair rows R from b+1
        S.col_off = (int64_t)items.size();
        for (int k = 0; k < nsub; ++k) {
          const int m = c->sd_host[k].nblk;
          if (b + 1 >= m || !L(k, b + 1, b)) continue;
          for (int R = 0; b + 1 + 2 * R < m; ++R) {
            const int r0 = b + 1 + 2 * R;
            if (L(k, r0, b) || L(k, r0 + 1, b)) items.push_back(make_int4(k, R, 0, 0));
          }
        }
        S.col_cnt = (int)((int64_t)items.size() - S.col_off);
        add_trsm(b + 1, &S.trsm_off[1], &S.trsm_cnt[1]);
      }
      S.trail_off = (int64_t)items.size();
      const int t0 = b + S.kb;
      for (int k = 0; k < nsub; ++k) {
        const int m = c->sd_host[k].nblk;
        if (t0 >= m) continue;
        // blocks i >= t0 reached by the step's panels
        std::vector<unsigned char> hit(m, 0);
        for (int i = t0; i < m; ++i)
          for (int p = b; p < b + S.kb; ++p) hit[i] |= L(k, i, p);
        auto upd = [&](int i, int j) {   // tile (i, j), i >= j, updated by a panel of the step
          if (i >= m || j >= m || i < j) return false;
          for (int p = b; p < b + S.kb; ++p)
            if (L(k, i, p) && L(k, j, p)) return true;
          return false;
        };
        if (prec == 1) {
          for (int R = 0; t0 + 2 * R < m; ++R)
            for (int C = 0; C <= R; ++C) {
              const int r0 = t0 + 2 * R, c0 = t0 + 2 * C;
              if (upd(r0, c0) || upd(r0 + 1, c0) || upd(r0, c0 + 1) || upd(r0 + 1, c0 + 1))
                items.push_back(make_int4(k, R, C, 0));
            }
        } else {
          for (int i = t0; i < m; ++i) {
            if (!hit[i]) continue;
            for (int j = t0; j <= i; ++j)
              if (upd(i, j)) items.push_back(make_int4(k, i, j, 0));
          }
        }
      }
      S.trail_cnt = (int)((int64_t)items.size() - S.trail_off);
      // the tiles of the next panels first (FP32: pair column 0, FP64: block
      // column t0), so that the next step's panel work can start after them
      // while the rest of the update runs on a second stream
      auto first = [&](const int4& it) { return prec == 1 ? it.z == 0 : it.z == t0; };
      std::stable_partition(items.begin() + S.trail_off, items.end(), first);
      S.trail_cnt0 = (int)std::count_if(items.begin() + S.trail_off, items.end(), first);
      P.steps.push_back(S);
      b += S.kb;
    }
    if (items.empty()) items.push_back(make_int4(0, 0, 0, 0));
    if (trsm.empty()) trsm.push_back(make_int2(0, 0));
    if ((r = dev_upload(c, &P.d_items, items)) != IETI_OK) return r;
    if ((r = dev_upload(c, &P.d_trsm, trsm)) != IETI_OK) return r;
    P.built = true;
  }
  // ---- nonzero tiles of every block row (ascending) and block column
  // (descending) of the factor, for the sweeps
  const int nb = c->blk_base[nsub];
  std::vector<int64_t> rp(nb + 1), cp(nb + 1);
  std::vector<int32_t> rc, cr;
  for (int k = 0; k < nsub; ++k) {
    const int m = c->sd_host[k].nblk;
    for (int b = 0; b < m; ++b) {
      rp[c->blk_base[k] + b] = (int64_t)rc.size();
      for (int j = 0; j < b; ++j)
        if (L(k, b, j)) rc.push_back(j);
      cp[c->blk_base[k] + b] = (int64_t)cr.size();
      for (int j = m - 1; j > b; --j)
        if (L(k, j, b)) cr.push_back(j);
    }
  }
  rp[nb] = (int64_t)rc.size();
  cp[nb] = (int64_t)cr.size();
  if (rc.empty()) rc.push_back(0);
  if (cr.empty()) cr.push_back(0);
  if ((r = dev_upload(c, &c->d_lrow_ptr, rp)) != IETI_OK) return r;
  if ((r = dev_upload(c, &c->d_lrow_col, rc)) != IETI_OK) return r;
  if ((r = dev_upload(c, &c->d_lcol_ptr, cp)) != IETI_OK) return r;
  if ((r = dev_upload(c, &c->d_lcol_row, cr)) != IETI_OK) return r;
  if ((r = dev_upload(c, &c->d_lflags, F)) != IETI_OK) return r;
  std::vector<int4> lt;
  for (int k = 0; k < nsub; ++k) {
    const int m = c->sd_host[k].nblk;
    for (int J = 0; J < m; ++J)
      for (int I = J; I < m; ++I)
        if (L(k, I, J)) lt.push_back(make_int4(k, I, J, 0));
  }
  c->n_ltiles = (int)lt.size();
  if (lt.empty()) lt.push_back(make_int4(0, 0, 0, 0));
  if ((r = dev_upload(c, &c->d_ltile_list, lt)) != IETI_OK) return r;
  if ((r = dev_upload(c, &c->d_tile_off, c->tile_off)) != IETI_OK) return r;
  int64_t nz = 0, tot = 0;
  for (int k = 0; k < nsub; ++k) {
    const int m = c->sd_host[k].nblk;
    tot += (int64_t)m * (m + 1) / 2;
  }
  for (unsigned char f : F) nz += f;
  c->lfill = tot ? (double)nz / (double)tot : 1.0;
  c->symb_ready = true;
  return IETI_OK;
}

}  // namespace ieti
