// Host sanitizer run of the geometry oracle (test infrastructure only): the
// test suite compiles this file with -fsanitize=address,undefined together
// with geom.cpp and runs it.  It drives every entry point of geom.cpp on a
// small random triangle soup, including the empty cases, and checks that the
// oracle's BVH agrees with its brute-force cast.  Prints OK on success.
#include "geom.cpp"

#include <cstdio>
#include <cstdlib>
#include <vector>

namespace {
uint64_t lcg_state = 0x2545F4914F6CDD1DULL;
float rnd(float lo, float hi) {  // inputs only: a plain 64-bit LCG
  lcg_state = lcg_state * 6364136223846793005ULL + 1442695040888963407ULL;
  return lo + (hi - lo) * (float)((lcg_state >> 40) * (1.0 / 16777216.0));
}
}  // namespace

int main() {
  const int n_tris = 300, n_rays = 2000, n_obj = 3;
  std::vector<float> verts(9 * n_tris);
  std::vector<int32_t> tris(3 * n_tris);
  for (int k = 0; k < n_tris; ++k) {
    const float cx = rnd(-3, 3), cy = rnd(-3, 3), cz = rnd(-3, 3);
    for (int j = 0; j < 3; ++j) {
      verts[9 * k + 3 * j] = cx + rnd(-0.5f, 0.5f);
      verts[9 * k + 3 * j + 1] = cy + rnd(-0.5f, 0.5f);
      verts[9 * k + 3 * j + 2] = cz + rnd(-0.5f, 0.5f);
      tris[3 * k + j] = 3 * k + j;
    }
  }
  std::vector<float> rays(8 * n_rays);
  for (int i = 0; i < n_rays; ++i) {
    float* r = &rays[8 * i];
    r[0] = rnd(-5, 5); r[1] = rnd(-5, 5); r[2] = rnd(-5, 5);
    float dx = rnd(-1, 1), dy = rnd(-1, 1), dz = rnd(-1, 1);
    if (i % 17 == 0) { dy = 0.f; dz = 0.f; dx = 1.f; }  // axis-parallel
    const float len = std::sqrt(dx * dx + dy * dy + dz * dz);
    r[4] = dx / len; r[5] = dy / len; r[6] = dz / len;
    r[3] = i % 5 == 0 ? 0.5f : 0.f;
    r[7] = i % 7 == 0 ? 2.f : std::numeric_limits<float>::infinity();
    if (i % 23 == 0) r[7] = r[3];  // empty segment
  }
  std::vector<uint8_t> occ(n_rays), occ2(n_rays);
  std::vector<float> th(n_rays), th2(n_rays);
  std::vector<int32_t> pr(n_rays), pr2(n_rays);
  oracle_brute_cast(verts.data(), tris.data(), n_tris, rays.data(), n_rays, occ.data(), th.data(), pr.data(), 2);
  void* h = oracle_bvh_build(verts.data(), tris.data(), n_tris);
  oracle_bvh_cast(h, verts.data(), tris.data(), rays.data(), n_rays, 1, occ2.data(), th2.data(), pr2.data(), 2);
  int bad = 0;
  for (int i = 0; i < n_rays; ++i) bad += occ[i] != occ2[i] || pr[i] != pr2[i] || (pr[i] >= 0 && th[i] != th2[i]);
  oracle_bvh_cast(h, verts.data(), tris.data(), rays.data(), n_rays, 0, occ2.data(), nullptr, nullptr, 2);
  for (int i = 0; i < n_rays; ++i) bad += occ[i] != occ2[i];
  if (oracle_bvh_node_count(h) < 1) ++bad;
  oracle_bvh_free(h);
  // empty scene and zero rays
  void* e = oracle_bvh_build(verts.data(), tris.data(), 0);
  oracle_bvh_cast(e, verts.data(), tris.data(), rays.data(), n_rays, 1, occ2.data(), th2.data(), pr2.data(), 1);
  for (int i = 0; i < n_rays; ++i) bad += occ2[i] != 0 || pr2[i] != -1;
  oracle_bvh_free(e);
  oracle_brute_cast(verts.data(), tris.data(), n_tris, rays.data(), 0, nullptr, nullptr, nullptr, 1);
  // pairs: objects are consecutive thirds of the soup
  std::vector<int64_t> first(n_obj), count(n_obj);
  for (int k = 0; k < n_obj; ++k) { first[k] = k * (n_tris / n_obj); count[k] = n_tris / n_obj; }
  const int nq = 3 * n_rays;
  std::vector<int32_t> rid(nq), ob(nq);
  for (int q = 0; q < nq; ++q) { rid[q] = q / 3; ob[q] = q % 3; }
  std::vector<uint8_t> hit(nq);
  std::vector<float> tq(nq);
  std::vector<int32_t> pq(nq);
  oracle_brute_pairs(verts.data(), tris.data(), first.data(), count.data(), rays.data(), rid.data(), ob.data(), nq,
                     hit.data(), 2);
  oracle_brute_pairs_closest(verts.data(), tris.data(), first.data(), count.data(), rays.data(), rid.data(),
                             ob.data(), nq, tq.data(), pq.data(), 2);
  for (int q = 0; q < nq; ++q) bad += (hit[q] != 0) != (pq[q] >= 0);
  const float box[6] = {-1, -1, -1, 1, 1, 1};
  for (int i = 0; i < n_rays; ++i) {
    float tin, tout, entry;
    oracle_slab(&rays[8 * i], box, &tin, &tout, &entry);
  }
  float t;
  const float v0[3] = {0, 0, 0}, v1[3] = {1, 0, 0}, v2[3] = {0, 1, 0};
  const float ray[8] = {0.25f, 0.25f, 1.f, 0.f, 0.f, 0.f, -1.f, 10.f};
  bad += oracle_mt_hit(ray, v0, v1, v2, &t) != 1 || t != 1.f;
  if (bad) {
    std::printf("MISMATCH %d\n", bad);
    return 1;
  }
  std::printf("OK\n");
  return 0;
}
