// Observation-graph preprocessing done once by ba_create: validation, the internal
// point and observation order, camera-major lists and the warp-tile / CTA-chunk
// decomposition used by the implicit Schur product.  Index bookkeeping only; no
// numerical step of the method runs here.
#include <algorithm>
#include <numeric>

#include "ba_internal.h"

namespace ba {


void build_graph(ba_problem* P, const int32_t* cam_idx_dev, const int32_t* pt_idx_dev) {
  const int n_c = P->n_c, n_p = P->n_p, n_o = P->n_o;
  std::vector<int32_t> cam(n_o), pt(n_o);
  if (n_o > 0) {
    BA_CUDA(cudaMemcpyAsync(cam.data(), cam_idx_dev, sizeof(int32_t) * n_o, cudaMemcpyDeviceToHost,
                            P->stream));
    BA_CUDA(cudaMemcpyAsync(pt.data(), pt_idx_dev, sizeof(int32_t) * n_o, cudaMemcpyDeviceToHost,
                            P->stream));
  }
  sync(P);
  for (int o = 0; o < n_o; ++o) {
    BA_REQUIRE(cam[o] >= 0 && cam[o] < n_c, BA_ERR_INVALID_ARG,
               "cam_idx[" + std::to_string(o) + "] out of range");
    BA_REQUIRE(pt[o] >= 0 && pt[o] < n_p, BA_ERR_INVALID_ARG,
               "pt_idx[" + std::to_string(o) + "] out of range");
  }
  // per caller point: observation count and first camera
  std::vector<int> cnt(n_p, 0), mincam(n_p, n_c);
  for (int o = 0; o < n_o; ++o) {
    cnt[pt[o]]++;
    mincam[pt[o]] = std::min(mincam[pt[o]], cam[o]);
  }
  // internal point order: observed points by (first camera, caller index); unobserved last
  std::vector<int> bucket(n_c + 2, 0);
  for (int p = 0; p < n_p; ++p) bucket[(cnt[p] ? mincam[p] : n_c) + 1]++;
  for (int i = 0; i <= n_c; ++i) bucket[i + 1] += bucket[i];
  std::vector<int> pt_user(n_p), pt_int(n_p);
  for (int p = 0; p < n_p; ++p) {
    int key = cnt[p] ? mincam[p] : n_c;
    int ip = bucket[key]++;
    pt_user[ip] = p;
    pt_int[p] = ip;
  }
  int n_p_obs = 0, max_pt_obs = 0;
  for (int p = 0; p < n_p; ++p) {
    n_p_obs += cnt[p] > 0;
    max_pt_obs = std::max(max_pt_obs, cnt[p]);
  }
  P->n_p_obs = n_p_obs;
  P->max_pt_obs = max_pt_obs;
  // observations grouped by internal point, sorted by camera inside each point
  std::vector<int32_t> pt_ptr(n_p + 1, 0);
  for (int ip = 0; ip < n_p; ++ip) pt_ptr[ip + 1] = pt_ptr[ip] + cnt[pt_user[ip]];
  std::vector<int32_t> fill(pt_ptr.begin(), pt_ptr.end() - 1);
  std::vector<int32_t> obs_user(n_o);
  for (int o = 0; o < n_o; ++o) obs_user[fill[pt_int[pt[o]]]++] = o;
  std::vector<int32_t> obs_cam(n_o), obs_ptu(n_o), obs_pt(n_o);
  for (int ip = 0; ip < n_p; ++ip) {
    auto b = obs_user.begin() + pt_ptr[ip], e = obs_user.begin() + pt_ptr[ip + 1];
    std::sort(b, e, [&](int a, int c) { return cam[a] != cam[c] ? cam[a] < cam[c] : a < c; });
    for (int k = pt_ptr[ip]; k < pt_ptr[ip + 1]; ++k) {
      obs_cam[k] = cam[obs_user[k]];
      obs_ptu[k] = pt_user[ip];
      obs_pt[k] = ip;
      BA_REQUIRE(k == pt_ptr[ip] || obs_cam[k] != obs_cam[k - 1], BA_ERR_INVALID_ARG,
                 "camera " + std::to_string(obs_cam[k]) + " observes point " +
                     std::to_string(pt_user[ip]) + " more than once");
    }
  }
  // camera-major lists (observations of a camera in increasing internal order)
  std::vector<int32_t> cam_ptr(n_c + 1, 0), cam_obs(n_o);
  for (int o = 0; o < n_o; ++o) cam_ptr[obs_cam[o] + 1]++;
  for (int c = 0; c < n_c; ++c) cam_ptr[c + 1] += cam_ptr[c];
  {
    std::vector<int32_t> f2(cam_ptr.begin(), cam_ptr.end() - 1);
    for (int o = 0; o < n_o; ++o) cam_obs[f2[obs_cam[o]]++] = o;
  }
  long long max_contrib = 0;
  for (int c = 0; c < n_c; ++c) {
    long long s = 0;
    for (int k = cam_ptr[c]; k < cam_ptr[c + 1]; ++k) {
      int ip = obs_pt[cam_obs[k]];
      s += pt_ptr[ip + 1] - pt_ptr[ip];
    }
    max_contrib = std::max(max_contrib, s);
  }
  P->max_row_contrib = (int)std::min<long long>(max_contrib, 1 << 30);

  // warp tiles: runs of whole points with at most 32 observations
  std::vector<int32_t> tile_pt;
  tile_pt.push_back(0);
  {
    int ip = 0;
    while (ip < n_p_obs) {
      int acc = cnt[pt_user[ip]];
      ++ip;
      if (acc <= 32)
        while (ip < n_p_obs && acc + cnt[pt_user[ip]] <= 32) acc += cnt[pt_user[ip++]];
      tile_pt.push_back(ip);
    }
  }
  const int n_tiles = (int)tile_pt.size() - 1;
  // per-tile descriptor for the Schur product: first observation, observation count,
  // first point and the mask of lanes that start a point (bit i: observation ob + i)
  std::vector<int4> tile_desc(std::max(n_tiles, 1));
  for (int t = 0; t < n_tiles; ++t) {
    const int p0 = tile_pt[t], p1 = tile_pt[t + 1];
    const int ob = pt_ptr[p0], nobs = pt_ptr[p1] - ob;
    unsigned mask = 1u;
    if (nobs <= 32)
      for (int p = p0; p < p1; ++p) mask |= 1u << (pt_ptr[p] - ob);
    tile_desc[t] = make_int4(ob, nobs, p0, (int)mask);
  }
  // per-tile camera order of the lanes, for the camera-side reduction of the FP32 Schur
  // product: byte j of tile t = (lane holding the j-th observation in camera order) |
  // 128 if position j starts a run of equal cameras; positions >= the observation
  // count map to themselves and start their own run
  std::vector<uint8_t> tile_perm((size_t)std::max(n_tiles, 1) * 32);
  for (int t = 0; t < n_tiles; ++t) {
    const int ob = tile_desc[t].x, nobs = tile_desc[t].y;
    int idx[32];
    for (int j = 0; j < 32; ++j) idx[j] = j;
    if (nobs <= 32)
      std::stable_sort(idx, idx + nobs, [&](int a, int b) { return obs_cam[ob + a] < obs_cam[ob + b]; });
    for (int j = 0; j < 32; ++j) {
      const bool head = nobs > 32 || j >= nobs || j == 0 || obs_cam[ob + idx[j]] != obs_cam[ob + idx[j - 1]];
      tile_perm[(size_t)t * 32 + j] = (uint8_t)(idx[j] | (head ? 128 : 0));
    }
  }
  // CTA chunks: contiguous tile ranges with about equal observation counts, a dozen per
  // SM so that CTAs looping over them stay balanced
  int want = std::max(1, std::min(P->n_sm * 12, n_tiles / 8));
  if (n_tiles == 0) want = 0;
  std::vector<int32_t> chunk_tile(1, 0), chunk_cam;
  if (n_tiles > 0) {
    long long total = n_o;
    int t = 0;
    for (int k = 1; k <= want; ++k) {
      long long target = total * k / want;
      while (t < n_tiles && pt_ptr[tile_pt[t + 1]] <= target) ++t;
      if (k == want) t = n_tiles;
      if (t > chunk_tile.back()) chunk_tile.push_back(t);
    }
    if (chunk_tile.back() != n_tiles) chunk_tile.push_back(n_tiles);
  }
  const int n_chunks = (int)chunk_tile.size() - 1;
  chunk_cam.resize(2 * std::max(n_chunks, 1), 0);
  for (int k = 0; k < n_chunks; ++k) {
    int lo = n_c, hi = -1;
    for (int o = pt_ptr[tile_pt[chunk_tile[k]]]; o < pt_ptr[tile_pt[chunk_tile[k + 1]]]; ++o) {
      lo = std::min(lo, obs_cam[o]);
      hi = std::max(hi, obs_cam[o]);
    }
    chunk_cam[2 * k] = lo;
    chunk_cam[2 * k + 1] = hi;
  }
  P->n_tiles = n_tiles;
  P->n_chunks = n_chunks;
  P->k3_window = std::max(1, std::min(n_c, 1024));
  P->ld = ((size_t)std::max(n_o, 1) + 31) / 32 * 32;
  P->ldp = ((size_t)std::max(n_p, 1) + 31) / 32 * 32;

  upload(P, P->obs_user, obs_user);
  upload(P, P->obs_cam, obs_cam);
  upload(P, P->obs_ptu, obs_ptu);
  upload(P, P->obs_pt, obs_pt);
  upload(P, P->pt_ptr, pt_ptr);
  upload(P, P->pt_user, pt_user);
  upload(P, P->cam_ptr, cam_ptr);
  upload(P, P->cam_obs, cam_obs);
  upload(P, P->tile_pt, tile_pt);
  upload(P, P->tile_desc, tile_desc);
  upload(P, P->tile_perm, tile_perm);
  upload(P, P->chunk_tile, chunk_tile);
  upload(P, P->chunk_cam, chunk_cam);
  sync(P);
}

}  // namespace ba
