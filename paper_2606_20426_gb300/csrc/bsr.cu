// Block-sparse (BSR, 3x3 blocks) layout of the Newton matrix, built once per
// env on the host from the fixed topology.
//
// Rows and columns are the free vertices; block (i, j) exists when i and j
// share a tet.  Every block keeps the list of element contributions
// (tet, corner a of i, corner b of j) in ascending tet order, and the list of
// contact contributions (contact vertex / edge / face holding both i and j,
// with their local corners) in kind-then-primitive order, so the per-Newton
// assembly is a fixed-order gather: no atomics, and the same sums whatever
// else runs in the batch.  Contact primitives lie on boundary faces of tets,
// so their vertex pairs are always blocks of the pattern.
//
// The entries themselves are stored in slices of 32 free rows (SELL-32, see
// EnvView::bsr_val): the PCG gives each lane of a warp one row of a slice,
// so the loads of block kk of the slice's rows are one coalesced access.
// On the structured tet meshes of the sensors the rows of a slice are
// nearly equally long (interior vertices have 15 blocks), so the slices add
// about 2 % unused slots.
#include <algorithm>
#include <vector>

#include "env.cuh"

namespace tc {

#define TC_TRY(x)                                  \
  do {                                             \
    if ((x) != cudaSuccess) return TC_ERR_CUDA;    \
  } while (0)

tc_status build_bsr(Env& env, const int32_t* tets, const int32_t* fixed_ids, int32_t nfixed) {
  Arena& a = env.arena;
  cudaStream_t s = env.stream;
  const int nv = env.nv, nt = env.nt;
  std::vector<uint8_t> fixed(nv, 0);
  for (int i = 0; i < nfixed; ++i)
    if (fixed_ids[i] >= 0 && fixed_ids[i] < nv) fixed[fixed_ids[i]] = 1;
  // --- pattern: sorted unique (row, col) pairs over free vertices
  std::vector<uint64_t> keys;
  keys.reserve(16 * (size_t)nt);
  for (int t = 0; t < nt; ++t) {
    const int32_t* v = tets + 4 * (size_t)t;
    for (int i = 0; i < 4; ++i) {
      if (fixed[v[i]]) continue;
      for (int j = 0; j < 4; ++j)
        if (!fixed[v[j]]) keys.push_back(((uint64_t)(uint32_t)v[i] << 32) | (uint32_t)v[j]);
    }
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  const int64_t nnzb = (int64_t)keys.size();
  if (nnzb >= (int64_t)1 << 31) return TC_ERR_CAPACITY;
  std::vector<int32_t> rp(nv + 1, 0), ci(nnzb), diag(nv, -1);
  for (int64_t k = 0; k < nnzb; ++k) {
    const int i = (int)(keys[k] >> 32), j = (int)(uint32_t)keys[k];
    rp[i + 1]++;
    ci[k] = j;
    if (i == j) diag[i] = (int32_t)k;
  }
  for (int i = 0; i < nv; ++i) rp[i + 1] += rp[i];
  // --- SELL-32 slices over the free (non-empty) rows
  std::vector<int32_t> free_v, free_of(nv, -1);
  for (int i = 0; i < nv; ++i)
    if (rp[i + 1] > rp[i]) {
      free_of[i] = (int32_t)free_v.size();
      free_v.push_back(i);
    }
  const int nfree = (int)free_v.size(), nsl = (nfree + 31) / 32;
  std::vector<int32_t> soff(nsl + 1, 0);
  for (int s = 0; s < nsl; ++s) {
    int w = 0;
    for (int f = 32 * s; f < std::min(nfree, 32 * s + 32); ++f) w = std::max(w, rp[free_v[f] + 1] - rp[free_v[f]]);
    if ((int64_t)soff[s] + 32 * (int64_t)w >= ((int64_t)1 << 31)) return TC_ERR_CAPACITY;
    soff[s + 1] = soff[s] + 32 * w;
  }
  const int nsell = soff[nsl];
  std::vector<int32_t> sci(nsell);
  for (int s = 0; s < nsl; ++s)
    for (int f = 32 * s; f < 32 * s + 32; ++f) {
      const int v = f < nfree ? free_v[f] : (nfree > 0 ? free_v[nfree - 1] : 0);
      const int len = f < nfree ? rp[v + 1] - rp[v] : 0;
      for (int kk = 0; kk < (soff[s + 1] - soff[s]) / 32; ++kk)
        sci[soff[s] + 32 * kk + (f & 31)] = kk < len ? ci[rp[v] + kk] : v;
    }
  auto slot = [&](int i, int j) -> int64_t {
    const int32_t* b = ci.data() + rp[i];
    const int32_t* e = ci.data() + rp[i + 1];
    const int32_t* f = std::lower_bound(b, e, j);
    return (f != e && *f == j) ? (int64_t)(f - ci.data()) : -1;
  };
  // --- element contributions, ascending tet order within each block
  std::vector<int32_t> eoff(nnzb + 1, 0);
  std::vector<int32_t> tslot(16 * (size_t)nt, -1);
  for (int t = 0; t < nt; ++t) {
    const int32_t* v = tets + 4 * (size_t)t;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        if (fixed[v[i]] || fixed[v[j]]) continue;
        const int64_t k = slot(v[i], v[j]);
        tslot[16 * (size_t)t + 4 * i + j] = (int32_t)k;
        eoff[k + 1]++;
      }
  }
  for (int64_t k = 0; k < nnzb; ++k) eoff[k + 1] += eoff[k];
  std::vector<int32_t> eidx(eoff[nnzb]);
  {
    std::vector<int32_t> cur(eoff.begin(), eoff.end() - 1);
    for (int t = 0; t < nt; ++t)
      for (int q = 0; q < 16; ++q) {
        const int32_t k = tslot[16 * (size_t)t + q];
        if (k >= 0) eidx[cur[k]++] = 16 * t + q;
      }
  }
  // --- contact contributions: vertex (3x3), edge (6x6), face (9x9) Hessians
  const int nvc = env.nvc, nec = env.nec, nfc = env.nfc;
  std::vector<int32_t> cverts(nvc), cedges(2 * (size_t)nec);
  if (nvc > 0) TC_TRY(cudaMemcpyAsync(cverts.data(), env.cverts, sizeof(int32_t) * nvc, cudaMemcpyDeviceToHost, s));
  if (nec > 0)
    TC_TRY(cudaMemcpyAsync(cedges.data(), env.cedges, sizeof(int32_t) * 2 * nec, cudaMemcpyDeviceToHost, s));
  TC_TRY(cudaStreamSynchronize(s));
  if (nvc >= (1 << 26) || nec >= (1 << 26) || nfc >= (1 << 26)) return TC_ERR_CAPACITY;
  std::vector<std::pair<int64_t, int32_t>> cc;  // (block, code) in emission order
  auto emit = [&](int kind, int prim, const int* vv, int nloc) {
    for (int i = 0; i < nloc; ++i)
      for (int j = 0; j < nloc; ++j) {
        if (fixed[vv[i]] || fixed[vv[j]]) continue;
        const int64_t k = slot(vv[i], vv[j]);
        if (k < 0) continue;  // not a tet pair (cannot happen for boundary primitives)
        cc.push_back({k, (int32_t)(((uint32_t)kind << 30) | ((uint32_t)i << 28) | ((uint32_t)j << 26) | (uint32_t)prim)});
      }
  };
  for (int p = 0; p < nvc; ++p) emit(0, p, &cverts[p], 1);
  for (int p = 0; p < nec; ++p) {
    const int vv[2] = {cedges[p], cedges[(size_t)nec + p]};
    emit(1, p, vv, 2);
  }
  for (int p = 0; p < nfc; ++p) {
    const int vv[3] = {env.h_cfaces[3 * (size_t)p], env.h_cfaces[3 * (size_t)p + 1], env.h_cfaces[3 * (size_t)p + 2]};
    emit(2, p, vv, 3);
  }
  std::stable_sort(cc.begin(), cc.end(),
                   [](const std::pair<int64_t, int32_t>& x, const std::pair<int64_t, int32_t>& y) { return x.first < y.first; });
  std::vector<int32_t> coff(nnzb + 1, 0), cidx(cc.size());
  for (size_t q = 0; q < cc.size(); ++q) {
    coff[cc[q].first + 1]++;
    cidx[q] = cc[q].second;
  }
  for (int64_t k = 0; k < nnzb; ++k) coff[k + 1] += coff[k];
  // --- upload
  env.nnzb = (int)nnzb;
  env.nfree = nfree;
  env.nsell = nsell;
  env.free_v = a.alloc<int32_t>(std::max(nfree, 1));
  env.free_of = a.alloc<int32_t>(nv);
  env.sell_off = a.alloc<int32_t>(nsl + 1);
  env.sell_ci = a.alloc<int32_t>(std::max(nsell, 1));
  if (!env.free_v || !env.free_of || !env.sell_off || !env.sell_ci) return TC_ERR_OOM;
  if (nfree > 0) TC_TRY(cudaMemcpyAsync(env.free_v, free_v.data(), sizeof(int32_t) * nfree, cudaMemcpyHostToDevice, s));
  TC_TRY(cudaMemcpyAsync(env.free_of, free_of.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice, s));
  TC_TRY(cudaMemcpyAsync(env.sell_off, soff.data(), sizeof(int32_t) * (nsl + 1), cudaMemcpyHostToDevice, s));
  if (nsell > 0) TC_TRY(cudaMemcpyAsync(env.sell_ci, sci.data(), sizeof(int32_t) * nsell, cudaMemcpyHostToDevice, s));
  env.bsr_rp = a.alloc<int32_t>(nv + 1);
  env.bsr_ci = a.alloc<int32_t>(nnzb);
  env.bsr_diag = a.alloc<int32_t>(nv);
  env.be_off = a.alloc<int32_t>(nnzb + 1);
  env.be_idx = a.alloc<int32_t>((int64_t)eidx.size());
  env.bc_off = a.alloc<int32_t>(nnzb + 1);
  env.bc_idx = a.alloc<int32_t>((int64_t)cidx.size());
  if (!env.bsr_rp || !env.bsr_ci || !env.bsr_diag || !env.be_off || !env.be_idx || !env.bc_off || !env.bc_idx)
    return TC_ERR_OOM;
  TC_TRY(cudaMemcpyAsync(env.bsr_rp, rp.data(), sizeof(int32_t) * (nv + 1), cudaMemcpyHostToDevice, s));
  if (nnzb > 0) TC_TRY(cudaMemcpyAsync(env.bsr_ci, ci.data(), sizeof(int32_t) * nnzb, cudaMemcpyHostToDevice, s));
  TC_TRY(cudaMemcpyAsync(env.bsr_diag, diag.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice, s));
  TC_TRY(cudaMemcpyAsync(env.be_off, eoff.data(), sizeof(int32_t) * (nnzb + 1), cudaMemcpyHostToDevice, s));
  if (!eidx.empty())
    TC_TRY(cudaMemcpyAsync(env.be_idx, eidx.data(), sizeof(int32_t) * eidx.size(), cudaMemcpyHostToDevice, s));
  TC_TRY(cudaMemcpyAsync(env.bc_off, coff.data(), sizeof(int32_t) * (nnzb + 1), cudaMemcpyHostToDevice, s));
  if (!cidx.empty())
    TC_TRY(cudaMemcpyAsync(env.bc_idx, cidx.data(), sizeof(int32_t) * cidx.size(), cudaMemcpyHostToDevice, s));
  // the host vectors go out of scope: wait for the copies
  TC_TRY(cudaStreamSynchronize(s));
  return TC_OK;
}

}  // namespace tc
