// Isomorphism-class tables (Sec. 4.3, Fig. 3a): every labelled pattern of k
// nodes is mapped to its class, so classifying a candidate is one lookup of
// its fill-in mask. The paper hashes every pattern under every relabeling;
// here the same map is a dense table indexed by the mask (16 entries for
// k=3, 2048 for k=4), built once on the host.
#include <algorithm>
#include <mutex>

#include "hm_internal.cuh"

namespace hm {
namespace {

struct Layout {
  int k = 0;
  int nsub = 0;
  int members[11][4];
  int size[11];
  uint32_t nodes[11];
};

// subsets with 2..k members, by size, then lexicographic
Layout make_layout(int k) {
  Layout L;
  L.k = k;
  for (int a = 0; a < k; ++a)
    for (int b = a + 1; b < k; ++b) {
      L.members[L.nsub][0] = a;
      L.members[L.nsub][1] = b;
      L.size[L.nsub] = 2;
      L.nodes[L.nsub++] = (1u << a) | (1u << b);
    }
  for (int a = 0; a < k; ++a)
    for (int b = a + 1; b < k; ++b)
      for (int c = b + 1; c < k; ++c) {
        L.members[L.nsub][0] = a;
        L.members[L.nsub][1] = b;
        L.members[L.nsub][2] = c;
        L.size[L.nsub] = 3;
        L.nodes[L.nsub++] = (1u << a) | (1u << b) | (1u << c);
      }
  if (k == 4) {
    for (int i = 0; i < 4; ++i) L.members[L.nsub][i] = i;
    L.size[L.nsub] = 4;
    L.nodes[L.nsub++] = 0xFu;
  }
  return L;
}

ClassTables make_tables(int k) {
  const Layout L = make_layout(k);
  // image of every subset bit under every relabeling
  std::vector<std::vector<int>> image;
  std::vector<int> p(k);
  for (int i = 0; i < k; ++i) p[i] = i;
  do {
    std::vector<int> img(L.nsub);
    for (int b = 0; b < L.nsub; ++b) {
      uint32_t mapped = 0;
      for (int i = 0; i < k; ++i)
        if (L.nodes[b] & (1u << i)) mapped |= 1u << p[i];
      img[b] = (int)(std::find(L.nodes, L.nodes + L.nsub, mapped) - L.nodes);
    }
    image.push_back(img);
  } while (std::next_permutation(p.begin(), p.end()));

  const uint32_t nmask = 1u << L.nsub;
  std::vector<uint32_t> canon_of(nmask);
  std::vector<uint8_t> conn(nmask);
  for (uint32_t m = 0; m < nmask; ++m) {
    uint32_t best = m;
    for (const auto& img : image) {
      uint32_t r = 0;
      for (int b = 0; b < L.nsub; ++b)
        if (m & (1u << b)) r |= 1u << img[b];
      best = std::min(best, r);
    }
    canon_of[m] = best;
    // connectivity: grow the component of node 0 through the subsets present
    uint32_t reach = 1u, prev = 0;
    while (reach != prev) {
      prev = reach;
      for (int b = 0; b < L.nsub; ++b)
        if ((m & (1u << b)) && (L.nodes[b] & reach)) reach |= L.nodes[b];
    }
    conn[m] = reach == (1u << k) - 1u;
  }
  ClassTables T;
  T.k = k;
  for (uint32_t m = 0; m < nmask; ++m)
    if (conn[m]) T.canon.push_back(canon_of[m]);
  std::sort(T.canon.begin(), T.canon.end());
  T.canon.erase(std::unique(T.canon.begin(), T.canon.end()), T.canon.end());
  T.ncls = (int)T.canon.size();
  T.lut.assign(nmask, 0xFF);
  for (uint32_t m = 0; m < nmask; ++m)
    if (conn[m])
      T.lut[m] = (uint8_t)(std::lower_bound(T.canon.begin(), T.canon.end(), canon_of[m]) -
                           T.canon.begin());
  for (uint32_t c : T.canon) {
    int mc = 0, cm = 0;
    for (int b = 0; b < L.nsub; ++b) {
      if (!(c & (1u << b))) continue;
      if (L.size[b] > mc) {
        mc = L.size[b];
        cm = 1;
      } else if (L.size[b] == mc) {
        ++cm;
      }
    }
    T.maxcard.push_back(mc);
    T.countmax.push_back(cm);
  }
  return T;
}

std::mutex g_lut_mu;
uint8_t* g_lut_dev[2][64] = {{nullptr}};

}  // namespace

const ClassTables& class_tables(int k) {
  static const ClassTables t3 = make_tables(3);
  static const ClassTables t4 = make_tables(4);
  return k == 3 ? t3 : t4;
}

const uint8_t* device_lut(int k) {
  int dev = 0;
  HM_CUDA(cudaGetDevice(&dev));
  HM_CHECK(dev >= 0 && dev < 64, HM_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_lut_mu);
  uint8_t*& p = g_lut_dev[k == 3 ? 0 : 1][dev];
  if (!p) {
    const ClassTables& T = class_tables(k);
    HM_CUDA(cudaMalloc((void**)&p, T.lut.size()));
    HM_CUDA(cudaMemcpy(p, T.lut.data(), T.lut.size(), cudaMemcpyHostToDevice));
  }
  return p;
}

}  // namespace hm

extern "C" {

int hm_num_classes(int order) {
  if (order != 3 && order != 4) return -1;
  return hm::class_tables(order).ncls;
}

hm_status hm_class_info(int order, int cls, uint32_t* canonical_mask, int32_t* maxcard,
                        int32_t* countmax) {
  return hm::guarded([&] {
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    const hm::ClassTables& T = hm::class_tables(order);
    HM_CHECK(cls >= 0 && cls < T.ncls, HM_EINVAL, "class id out of range");
    if (canonical_mask) *canonical_mask = T.canon[cls];
    if (maxcard) *maxcard = T.maxcard[cls];
    if (countmax) *countmax = T.countmax[cls];
  });
}

hm_status hm_class_of_mask(int order, uint32_t mask, int32_t* cls) {
  return hm::guarded([&] {
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    const hm::ClassTables& T = hm::class_tables(order);
    HM_CHECK(mask < T.lut.size(), HM_EINVAL, "mask out of range");
    HM_CHECK(cls != nullptr, HM_EINVAL, "cls is NULL");
    *cls = T.lut[mask] == 0xFF ? -1 : (int32_t)T.lut[mask];
  });
}

}  // extern "C"
