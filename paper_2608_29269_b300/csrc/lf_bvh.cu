// Two-level LBVH build and refit (one BLAS per object, Eq. 2), the rigid
// object transform, and the environment importance-sampling tables.
#include <climits>

#include "lf_kernels.h"

namespace lf {

// ---------------------------------------------------------------- AABB + bounds
// Support ellipse of surfel i at radius R = sqrt(support_r2): in axis k its
// half extent is R * sqrt((s_u tu_k)^2 + (s_v tv_k)^2).  Boxes are padded by a
// small relative margin so that FP32 slab tests never miss an accepted hit.
__device__ __forceinline__ void surfel_box(const SceneDev& s, int i, float R, float3& lo, float3& hi) {
  const float su = s.scale[2 * i], sv = s.scale[2 * i + 1];
  float m[3], e[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    m[k] = s.mu[3 * i + k];
    const float a = su * s.tu[3 * i + k], b = sv * s.tv[3 * i + k];
    e[k] = R * sqrtf(a * a + b * b);
  }
  float p0 = 1e-5f * (1.0f + fabsf(m[0]) + e[0]), p1 = 1e-5f * (1.0f + fabsf(m[1]) + e[1]),
        p2 = 1e-5f * (1.0f + fabsf(m[2]) + e[2]);
  lo = f3(m[0] - e[0] - p0, m[1] - e[1] - p1, m[2] - e[2] - p2);
  hi = f3(m[0] + e[0] + p0, m[1] + e[1] + p1, m[2] + e[2] + p2);
}

__device__ __forceinline__ int ordered(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float unordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// Centroid bounds per object: grid.y = object, blocks stride over its range.
__global__ void k_object_bounds(SceneDev s, const int* __restrict__ offsets, int* __restrict__ bounds) {
  const int obj = blockIdx.y;
  const int beg = offsets[obj], end = offsets[obj + 1];
  float lo[3] = {BIG_F, BIG_F, BIG_F}, hi[3] = {-BIG_F, -BIG_F, -BIG_F};
  for (int i = beg + blockIdx.x * blockDim.x + threadIdx.x; i < end; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float v = s.mu[3 * i + k];
      lo[k] = fminf(lo[k], v);
      hi[k] = fmaxf(hi[k], v);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
    }
  }
  if ((threadIdx.x & 31) == 0 && end > beg) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicMin(bounds + 6 * obj + k, ordered(lo[k]));
      atomicMax(bounds + 6 * obj + 3 + k, ordered(hi[k]));
    }
  }
}

__global__ void k_bounds_init(int* bounds, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) bounds[i] = (i % 6) < 3 ? ordered(BIG_F) : ordered(-BIG_F);
}

__device__ __forceinline__ unsigned spread10(unsigned v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ int object_of(const int* offsets, int n_obj, int i) {
  int lo = 0, hi = n_obj - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// 30-bit Morton code of the surfel centre in its object's centroid bounds.
__global__ void k_morton(SceneDev s, const int* __restrict__ offsets, int n_obj, const int* __restrict__ bounds,
                         unsigned* __restrict__ keys, unsigned* __restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const int obj = object_of(offsets, n_obj, i);
  unsigned c[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float lo = unordered(bounds[6 * obj + k]), hi = unordered(bounds[6 * obj + 3 + k]);
    const float ext = hi - lo;
    float u = ext > 0.0f ? (s.mu[3 * i + k] - lo) / ext : 0.5f;
    u = fminf(fmaxf(u, 0.0f), 1.0f);
    c[k] = min(1023u, (unsigned)(u * 1024.0f));
  }
  keys[i] = (spread10(c[0]) << 2) | (spread10(c[1]) << 1) | spread10(c[2]);
  vals[i] = (unsigned)i;
}

// ---------------------------------------------------------------- radix sort
// One stable LSD pass over 8-bit digits: per-tile histograms, a global
// digit-major exclusive scan, and a scatter that ranks equal digits within a
// warp with __match_any_sync and across warps with per-warp counters.
constexpr int RS_THREADS = 256, RS_ITEMS = 16, RS_TILE = RS_THREADS * RS_ITEMS, RS_WARPS = RS_THREADS / 32;

__device__ __forceinline__ unsigned rs_digit(unsigned key, unsigned val, int shift, const int* offsets, int n_obj) {
  if (shift < 0) return (unsigned)object_of(offsets, n_obj, (int)val);  // object pass
  return (key >> shift) & 255u;
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const unsigned* __restrict__ keys,
                                                           const unsigned* __restrict__ vals, int n, int shift,
                                                           const int* offsets, int n_obj, unsigned* counts,
                                                           int n_tiles) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * RS_TILE;
  for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
    const int i = base + k;
    if (i < n) atomicAdd(&h[rs_digit(keys[i], vals[i], shift, offsets, n_obj)], 1u);
  }
  __syncthreads();
  counts[threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of counts[256 * n_tiles] in one block (digit-major order).
__global__ void __launch_bounds__(1024) k_radix_scan(unsigned* counts, int total) {
  __shared__ unsigned part[1024];
  const int per = (total + 1023) / 1024;
  const int beg = threadIdx.x * per, end = min(total, beg + per);
  unsigned s = 0;
  for (int i = beg; i < end; ++i) s += counts[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    unsigned v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned run = part[threadIdx.x] - s;
  for (int i = beg; i < end; ++i) {
    unsigned c = counts[i];
    counts[i] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const unsigned* __restrict__ keys_in,
                                                              const unsigned* __restrict__ vals_in,
                                                              unsigned* __restrict__ keys_out,
                                                              unsigned* __restrict__ vals_out, int n, int shift,
                                                              const int* offsets, int n_obj,
                                                              const unsigned* __restrict__ offs, int n_tiles) {
  __shared__ unsigned cnt[RS_WARPS][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < RS_WARPS * 256; k += RS_THREADS) (&cnt[0][0])[k] = 0;
  __syncthreads();
  const int base = blockIdx.x * RS_TILE + warp * (RS_ITEMS * 32);
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned pos[RS_ITEMS], dig[RS_ITEMS], key[RS_ITEMS], val[RS_ITEMS];
#pragma unroll
  for (int it = 0; it < RS_ITEMS; ++it) {
    const int i = base + it * 32 + lane;
    const bool valid = i < n;
    key[it] = valid ? keys_in[i] : 0u;
    val[it] = valid ? vals_in[i] : 0u;
    const unsigned d = valid ? rs_digit(key[it], val[it], shift, offsets, n_obj) : 256u;
    dig[it] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank = __popc(peers & lt_mask);
    const unsigned before = valid ? cnt[warp][d] : 0u;
    __syncwarp();
    if (valid && rank == 0) cnt[warp][d] = before + __popc(peers);
    __syncwarp();
    pos[it] = before + rank;
  }
  __syncthreads();
  {  // exclusive prefix over warps, one digit per thread
    const int d = threadIdx.x;
    unsigned run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      unsigned c = cnt[w][d];
      cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < RS_ITEMS; ++it) {
    const int i = base + it * 32 + lane;
    if (i < n) {
      const unsigned d = dig[it];
      const unsigned dst = offs[d * n_tiles + blockIdx.x] + cnt[warp][d] + pos[it];
      keys_out[dst] = key[it];
      vals_out[dst] = val[it];
    }
  }
}

// ---------------------------------------------------------------- Karras hierarchy
// Longest common prefix of keys i and j of one object (duplicates ordered by
// index), -1 outside [0, n).
__device__ __forceinline__ int delta(const unsigned* k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  const unsigned a = k[i], b = k[j];
  if (a == b) return 32 + __clz((unsigned)(i ^ j));
  return __clz(a ^ b);
}

__global__ void k_hierarchy(const unsigned* __restrict__ skeys, const int* __restrict__ leaf_off,
                            const int* __restrict__ node_off, int n_obj, int n_nodes_total,
                            float4* __restrict__ nodes, int* __restrict__ leaf_parent,
                            int* __restrict__ node_parent, int2* __restrict__ node_range) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_nodes_total) return;
  const int obj = object_of(node_off, n_obj, g);
  const int i = g - node_off[obj];
  const int lb = leaf_off[obj], n = leaf_off[obj + 1] - lb, nb = node_off[obj];
  const unsigned* k = skeys + lb;
  const int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
  const int dmin = delta(k, n, i, i - d);
  int lmax = 2;
  while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
  const int j = i + l * d;
  const int dnode = delta(k, n, i, j);
  int s = 0;
  for (int div = 2;; div <<= 1) {
    const int t = (l + div - 1) / div;
    if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
    if (t <= 1) break;
  }
  const int gamma = i + s * d + min(d, 0);
  const int left = (min(i, j) == gamma) ? ~gamma : gamma;
  const int right = (max(i, j) == gamma + 1) ? ~(gamma + 1) : gamma + 1;
  nodes[4 * (nb + i) + 3] = make_float4(__int_as_float(left), __int_as_float(right), 0.f, 0.f);
  node_range[nb + i] = make_int2(min(i, j), abs(i - j) + 1);  // first leaf, leaf count
  if (left < 0) leaf_parent[lb + gamma] = (i << 1) | 0; else node_parent[nb + gamma] = (i << 1) | 0;
  if (right < 0) leaf_parent[lb + gamma + 1] = (i << 1) | 1; else node_parent[nb + gamma + 1] = (i << 1) | 1;
  if (i == 0) node_parent[nb] = -1;
}

// ---------------------------------------------------------------- pack + fit
__device__ __forceinline__ void write_child_box(float4* node, int side, float3 lo, float3 hi) {
  float* f = reinterpret_cast<float*>(node);
  const int b = side == 0 ? 0 : 6;
  __stcg(f + b + 0, lo.x); __stcg(f + b + 1, lo.y); __stcg(f + b + 2, lo.z);
  __stcg(f + b + 3, hi.x); __stcg(f + b + 4, hi.y); __stcg(f + b + 5, hi.z);
}

// One thread per leaf of the selected objects: pack the surfel's records,
// compute its box and propagate boxes to the root; the second child to
// arrive at a node forms the union (atomic visit counter per node).
//
// Index bases: the leaves, node links and sorted ids are those of the build
// (global numbering); a.leaf_base / a.node_base / a.id_base / a.inst_base are
// subtracted when writing records, nodes, flags and the instance entry and
// when reading the raw attributes, so the same kernel fits both the
// context's own storage (bases 0) and an object-local copy (a served version).
__global__ void k_pack_fit(SceneDev s, FitArgs a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n_leaves) return;
  const int L = a.first_leaf + g;
  const int obj = object_of(a.leaf_off, a.n_obj, L);
  const int lb = a.leaf_off[obj], n = a.leaf_off[obj + 1] - lb, nb = a.node_off[obj];
  const int id = (int)a.sorted_ids[L];
  const int i = id - a.id_base;  // raw attribute index
  const int Lw = L - a.leaf_base, nbw = nb - a.node_base;
  // pack
  const float su = s.scale[2 * i], sv = s.scale[2 * i + 1];
  const float3 mu = f3(s.mu[3 * i], s.mu[3 * i + 1], s.mu[3 * i + 2]);
  const float3 tu = f3(s.tu[3 * i], s.tu[3 * i + 1], s.tu[3 * i + 2]);
  const float3 tv = f3(s.tv[3 * i], s.tv[3 * i + 1], s.tv[3 * i + 2]);
  // unit normal tu x tv, normalised in FP64 (axis-aligned planes stay exact)
  const double cx = (double)tu.y * tv.z - (double)tu.z * tv.y, cy = (double)tu.z * tv.x - (double)tu.x * tv.z,
               cz = (double)tu.x * tv.y - (double)tu.y * tv.x;
  const double cl = sqrt(cx * cx + cy * cy + cz * cz);
  const float3 nh = f3((float)(cx / cl), (float)(cy / cl), (float)(cz / cl));
  const float3 ax = f3(tu.x / su, tu.y / su, tu.z / su), bx = f3(tv.x / sv, tv.y / sv, tv.z / sv);
  float4* rec = a.geo + (size_t)GEO * (lb - a.leaf_base) + (L - lb);  // the object's planes of n quads
  rec[0] = make_float4(mu.x, mu.y, mu.z, nh.x);
  rec[(size_t)n] = make_float4(nh.y, nh.z, ax.x, ax.y);
  rec[2 * (size_t)n] = make_float4(ax.z, bx.x, bx.y, bx.z);
  rec[3 * (size_t)n] = make_float4(s.opacity[i], __int_as_float(id), s.roughness[i], 0.0f);
  a.mat[Lw] = make_float4(s.albedo[3 * i], s.albedo[3 * i + 1], s.albedo[3 * i + 2], s.metallic[i]);
  float3 lo, hi;
  surfel_box(s, i, a.R, lo, hi);
  Inst* inst = a.insts + (obj - a.inst_base);
  if (n == 1) {
    inst->lo[0] = lo.x; inst->lo[1] = lo.y; inst->lo[2] = lo.z;
    inst->hi[0] = hi.x; inst->hi[1] = hi.y; inst->hi[2] = hi.z;
    return;
  }
  int link = a.leaf_parent[L];
  for (int guard = 0; guard < n; ++guard) {
    if (link < 0 || (link >> 1) >= n - 1) {  // malformed hierarchy: leave the boxes, report
      report(a.status, LF_ERR_INVALID);
      return;
    }
    const int p = link >> 1, side = link & 1;
    float4* node = a.nodes + 4 * (nbw + p);
    write_child_box(node, side, lo, hi);
    __threadfence();
    if (atomicAdd(a.flags + nbw + p, 1) == 0) return;
    __threadfence();
    const float* f = reinterpret_cast<const float*>(node);
    lo = f3(fminf(__ldcg(f + 0), __ldcg(f + 6)), fminf(__ldcg(f + 1), __ldcg(f + 7)), fminf(__ldcg(f + 2), __ldcg(f + 8)));
    hi = f3(fmaxf(__ldcg(f + 3), __ldcg(f + 9)), fmaxf(__ldcg(f + 4), __ldcg(f + 10)), fmaxf(__ldcg(f + 5), __ldcg(f + 11)));
    if (p == 0) {
      inst->lo[0] = lo.x; inst->lo[1] = lo.y; inst->lo[2] = lo.z;
      inst->hi[0] = hi.x; inst->hi[1] = hi.y; inst->hi[2] = hi.z;
      return;
    }
    link = a.node_parent[nb + p];
  }
  report(a.status, LF_ERR_INVALID);
}

// ---------------------------------------------------------------- wide BVH
// The binary BLAS of each object is collapsed into a WIDE-ary tree whose
// nodes are traversed by WIDE lanes at once (one child slot per lane).  A wide
// node starts from a binary node's two children and repeatedly replaces the
// child with the largest box surface (the one rays enter most often) by its
// own two children, while fewer than WIDE children are held and that child has
// more than WLEAF leaves.  A child with at most WLEAF leaves becomes a leaf
// slot (its surfels are consecutive in leaf order); a larger one becomes a
// wide node of its own.  The collapse runs once per build, after the first
// fit; a refit keeps the topology and only copies boxes (k_wide_boxes) --
// a rigid motion moves every box of an object together, so the choices stay
// as good.  A wide node that is not full holds only
// leaf slots and covers more than WLEAF surfels; with I nodes, at most
// n / (WLEAF + 1) of them not full and n leaf slots, I (WIDE - 1) <= n +
// (WIDE - 2) n / (WLEAF + 1), the capacity wide_capacity() allocates.
//
// Topology: one block per object, level by level (breadth first); children
// get consecutive indices in item order (block-wide scan), so the layout is
// deterministic.  wsrc[slot] = binary parent (object-local) * 2 + side of the
// slot's box; -1 for an empty slot.
constexpr int COLLAPSE_THREADS = 128;

__global__ void __launch_bounds__(COLLAPSE_THREADS) k_collapse(WideArgs a) {
  __shared__ int s_scan[COLLAPSE_THREADS];
  const int obj = a.first_obj + blockIdx.x;
  const int n = a.leaf_off[obj + 1] - a.leaf_off[obj];
  if (n <= WLEAF) return;  // the root is a leaf slot held by the instance
  const int nb = a.node_off[obj];                      // binary nodes, global numbering (ranges)
  const int wb = a.wnode_off[obj];                     // wide nodes, global numbering
  const int cap = a.wnode_off[obj + 1] - wb;
  const float4* bnodes = a.nodes + 4 * (size_t)(nb - a.node_base);
  float4* wn = a.wnodes + WNODE_Q * (size_t)(wb - a.wnode_base);
  int* wsrc = a.wsrc + WIDE * (size_t)(wb - a.wsrc_base);
  int* queue = a.wqueue + (wb - a.wnode_base);
  if (threadIdx.x == 0) queue[0] = 0;
  __syncthreads();
  int level_begin = 0, level_end = 1, total = 1;
  bool overflow = false;
  while (level_begin < level_end && !overflow) {
    for (int chunk = level_begin; chunk < level_end; chunk += COLLAPSE_THREADS) {
      const int item = chunk + threadIdx.x;
      const bool valid = item < level_end;
      int code[WIDE], cnt[WIDE], src[WIDE];
      float prio[WIDE];
      int nc = 0, n_int = 0;
      // expansion priority of a child: the surface of its box (stored in its
      // binary parent), half of it
      auto priority = [&](int parent, int side) -> float {
        const float* f = reinterpret_cast<const float*>(bnodes + 4 * parent) + (side ? 6 : 0);
        const float dx = f[3] - f[0], dy = f[4] - f[1], dz = f[5] - f[2];
        return dx * dy + dy * dz + dz * dx;
      };
      if (valid) {
        const int b = queue[item];
        const float4 f = bnodes[4 * b + 3];
        const int cl = __float_as_int(f.x), cr = __float_as_int(f.y);
        code[0] = cl; src[0] = 2 * b + 0; cnt[0] = cl >= 0 ? a.node_range[nb + cl].y : 1;
        code[1] = cr; src[1] = 2 * b + 1; cnt[1] = cr >= 0 ? a.node_range[nb + cr].y : 1;
        prio[0] = priority(b, 0);
        prio[1] = priority(b, 1);
        nc = 2;
        while (nc < WIDE) {
          int best = -1;
          for (int c = 0; c < nc; ++c)
            if (code[c] >= 0 && cnt[c] > WLEAF && (best < 0 || prio[c] > prio[best])) best = c;
          if (best < 0) break;
          const int e = code[best];
          const float4 g = bnodes[4 * e + 3];
          const int el = __float_as_int(g.x), er = __float_as_int(g.y);
          code[best] = el; src[best] = 2 * e + 0; cnt[best] = el >= 0 ? a.node_range[nb + el].y : 1;
          code[nc] = er; src[nc] = 2 * e + 1; cnt[nc] = er >= 0 ? a.node_range[nb + er].y : 1;
          prio[best] = priority(e, 0);
          prio[nc] = priority(e, 1);
          ++nc;
        }
        for (int c = 0; c < nc; ++c) n_int += (code[c] >= 0 && cnt[c] > WLEAF) ? 1 : 0;
      }
      // exclusive scan of n_int over the chunk (item order)
      s_scan[threadIdx.x] = n_int;
      __syncthreads();
      for (int off = 1; off < COLLAPSE_THREADS; off <<= 1) {
        const int v = threadIdx.x >= off ? s_scan[threadIdx.x - off] : 0;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
      }
      const int chunk_total = s_scan[COLLAPSE_THREADS - 1];
      int next = total + s_scan[threadIdx.x] - n_int;
      if (total + chunk_total > cap) {
        overflow = true;  // uniform: every thread read the same scan total
      } else if (valid) {
        float4* node = wn + WNODE_Q * (size_t)item;
        for (int c = 0; c < WIDE; ++c) {
          int cd = INT_MIN, ct = 0, sr = -1;
          if (c < nc) {
            sr = src[c];
            if (code[c] >= 0 && cnt[c] > WLEAF) {
              cd = next;
              queue[next++] = code[c];
            } else {
              cd = ~(code[c] >= 0 ? a.node_range[nb + code[c]].x : ~code[c]);
              ct = cnt[c];
            }
          }
#if LF_WIDE_FP16
          const unsigned word = cd == INT_MIN ? WSLOT_EMPTY
                                : cd >= 0   ? (unsigned)cd
                                            : (0x80000000u | ((unsigned)(ct - 1) << 24) | (unsigned)~cd);
          reinterpret_cast<uint4*>(node)[1 + c] = make_uint4(0u, 0u, 0u, word);
#else
          node[c] = make_float4(1.0f, 1.0f, 1.0f, __int_as_float(cd));
          node[WIDE + c] = make_float4(-1.0f, -1.0f, -1.0f, __int_as_float(ct));
#endif
          wsrc[WIDE * item + c] = sr;
        }
      }
      total += chunk_total;
      __syncthreads();
    }
    level_begin = level_end;
    level_end = total;
  }
  if (overflow && threadIdx.x == 0) report(a.status, LF_ERR_INVALID);
}

// Box of every wide slot from the binary node holding it (build and refit).
#if LF_WIDE_FP16
// Compressed slots: one warp per wide node (slots of a node are WIDE
// consecutive threads; first_slot and n_slots are multiples of WIDE).  The
// node's centre is the centre of the union of its slot boxes; each corner is
// stored as an FP16 offset from it, rounded down (lo) or up (hi) after a
// subtraction rounded the same way, so the decoded box contains the slot's
// FP32 box.
__device__ __forceinline__ unsigned pack_h2(__half lo_half, __half hi_half) {
  return (unsigned)__half_as_ushort(lo_half) | ((unsigned)__half_as_ushort(hi_half) << 16);
}
#endif

__global__ void k_wide_boxes(WideArgs a, int n_slots) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_slots) return;
  const int slot = a.first_slot + k;
  const int sr = a.wsrc[slot - WIDE * a.wsrc_base];
  const int local = slot - WIDE * a.wnode_base;  // node * WIDE + c in the storage
#if LF_WIDE_FP16
  static_assert(WIDE == 32, "one warp per wide node");
  float b[6] = {BIG_F, BIG_F, BIG_F, -BIG_F, -BIG_F, -BIG_F};
  if (sr >= 0) {
    const int obj = object_of(a.wnode_off, a.n_obj_total, slot / WIDE);
    const int nb = a.node_off[obj] - a.node_base;
    const float* f = reinterpret_cast<const float*>(a.nodes + 4 * (size_t)(nb + (sr >> 1))) + ((sr & 1) ? 6 : 0);
#pragma unroll
    for (int q = 0; q < 6; ++q) b[q] = f[q];
  }
  float u[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) u[q] = b[q];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      u[q] = fminf(u[q], __shfl_xor_sync(0xffffffffu, u[q], off));
      u[q + 3] = fmaxf(u[q + 3], __shfl_xor_sync(0xffffffffu, u[q + 3], off));
    }
  const float cx = 0.5f * (u[0] + u[3]), cy = 0.5f * (u[1] + u[4]), cz = 0.5f * (u[2] + u[5]);
  float4* node = a.wnodes + WNODE_Q * (size_t)(local / WIDE);
  if ((local % WIDE) == 0) node[0] = make_float4(cx, cy, cz, 0.0f);
  if (sr < 0) return;
  const __half lx = __float2half_rd(__fsub_rd(b[0], cx)), ly = __float2half_rd(__fsub_rd(b[1], cy)),
               lz = __float2half_rd(__fsub_rd(b[2], cz));
  const __half hx = __float2half_ru(__fsub_ru(b[3], cx)), hy = __float2half_ru(__fsub_ru(b[4], cy)),
               hz = __float2half_ru(__fsub_ru(b[5], cz));
  uint4* w = reinterpret_cast<uint4*>(node) + 1 + (local % WIDE);
  const unsigned word = w->w;
  *w = make_uint4(pack_h2(lx, ly), pack_h2(lz, hx), pack_h2(hy, hz), word);
#else
  if (sr < 0) return;
  const int obj = object_of(a.wnode_off, a.n_obj_total, slot / WIDE);
  const int nb = a.node_off[obj] - a.node_base;
  const float* f = reinterpret_cast<const float*>(a.nodes + 4 * (size_t)(nb + (sr >> 1)));
  const int o = (sr & 1) ? 6 : 0;
  float4* w = a.wnodes + 2 * (size_t)WIDE * (local / WIDE) + (local % WIDE);
  const float4 p = w[0], q = w[WIDE];
  w[0] = make_float4(f[o + 0], f[o + 1], f[o + 2], p.w);
  w[WIDE] = make_float4(f[o + 3], f[o + 4], f[o + 5], q.w);
#endif
}

// ---------------------------------------------------------------- rigid transform
// Eq. 2 on one object's surfels: mu <- R mu + t, tu <- R tu, tv <- R tv.
// Each component is ((R0 x0 + R1 x1) + R2 x2) (+ t) in FP64, where every
// product of two FP32 values is exact, rounded once to FP32: the result does
// not depend on FMA contraction, so any FP64 evaluation in this order gives
// the same bits.
__global__ void k_rigid(SceneDev s, int beg, int end, Mat34 T) {
  const int i = beg + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= end) return;
  const double m[3] = {s.mu[3 * i], s.mu[3 * i + 1], s.mu[3 * i + 2]};
  const double u[3] = {s.tu[3 * i], s.tu[3 * i + 1], s.tu[3 * i + 2]};
  const double v[3] = {s.tv[3 * i], s.tv[3 * i + 1], s.tv[3 * i + 2]};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double R0 = T.R[3 * r], R1 = T.R[3 * r + 1], R2 = T.R[3 * r + 2];
    s.mu[3 * i + r] = __double2float_rn(__dadd_rn(__dadd_rn(__dadd_rn(R0 * m[0], R1 * m[1]), R2 * m[2]), (double)T.t[r]));
    s.tu[3 * i + r] = __double2float_rn(__dadd_rn(__dadd_rn(R0 * u[0], R1 * u[1]), R2 * u[2]));
    s.tv[3 * i + r] = __double2float_rn(__dadd_rn(__dadd_rn(R0 * v[0], R1 * v[1]), R2 * v[2]));
  }
}

__global__ void k_material(SceneDev s, int beg, int end, float3 rgb, int set_rgb, float metal, float rough) {
  const int i = beg + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= end) return;
  if (set_rgb) { s.albedo[3 * i] = rgb.x; s.albedo[3 * i + 1] = rgb.y; s.albedo[3 * i + 2] = rgb.z; }
  if (metal >= 0.0f) s.metallic[i] = metal;
  if (rough >= 0.0f) s.roughness[i] = rough;
}

// ---------------------------------------------------------------- environment tables
// Texel weight (Rec.709 luminance + 1e-6) * sin(theta at the row centre) in
// FP64 with explicit rounding (no contraction); sequential sums per row.
// One block per row.  The texel weights w_c = (lum + 1e-6) sin(theta) are
// formed in parallel into shared memory, chunk by chunk (coalesced loads);
// one thread sums them in column order (the same FP64 operations, in the
// same order, as a single thread walking the row), and the pmf / cdf
// divisions run in parallel again.
constexpr int ENV_T = 256;    // threads per row block
constexpr int ENV_CH = 1024;  // texels per shared-memory chunk

__device__ __forceinline__ double texel_weight(const float* t, double st) {
  double lum = __dadd_rn(__dmul_rn(0.2126, (double)t[0]), __dmul_rn(0.7152, (double)t[1]));
  lum = __dadd_rn(lum, __dmul_rn(0.0722, (double)t[2]));
  lum = __dadd_rn(lum, 1e-6);
  return __dmul_rn(lum, st);
}

// The FP64 CDF value v goes out as the FP32 pair (hi, lo): hi = v rounded,
// lo = v - hi rounded, so a sampler can place a uniform inside its texel to
// FP64 accuracy while it searches the FP32 table.
__device__ __forceinline__ void put_cdf(float* hi, float* lo, size_t i, double v) {
  const float h = (float)v;
  hi[i] = h;
  lo[i] = (float)__dsub_rn(v, (double)h);
}

__global__ void __launch_bounds__(ENV_T) k_env_rows(const float* __restrict__ rgb, const double* __restrict__ sin_row,
                                                    int H, int W, double* __restrict__ rowsum,
                                                    float* __restrict__ pmf_col, float* __restrict__ cdf_col,
                                                    float* __restrict__ cdf_col_lo) {
  __shared__ double s_w[ENV_CH], s_p[ENV_CH];
  __shared__ double s_acc;
  const int r = blockIdx.x;
  if (r >= H) return;  // uniform over the block
  const double st = sin_row[r];
  const float* row = rgb + 3 * (size_t)r * W;
  if (threadIdx.x == 0) s_acc = 0.0;
  // pass 1: the row sum, in column order
  for (int c0 = 0; c0 < W; c0 += ENV_CH) {
    const int n = min(ENV_CH, W - c0);
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += ENV_T) s_w[c] = texel_weight(row + 3 * (size_t)(c0 + c), st);
    __syncthreads();
    if (threadIdx.x == 0) {
      double acc = s_acc;
      for (int c = 0; c < n; ++c) acc = __dadd_rn(acc, s_w[c]);
      s_acc = acc;
    }
  }
  __syncthreads();
  const double acc = s_acc;
  if (threadIdx.x == 0) rowsum[r] = acc;
  // pass 2: the column cdf (prefix sums in column order) and pmf
  double pc = 0.0;  // running prefix, held by thread 0
  for (int c0 = 0; c0 < W; c0 += ENV_CH) {
    const int n = min(ENV_CH, W - c0);
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += ENV_T) s_w[c] = texel_weight(row + 3 * (size_t)(c0 + c), st);
    __syncthreads();
    if (threadIdx.x == 0)
      for (int c = 0; c < n; ++c) {
        pc = __dadd_rn(pc, s_w[c]);
        s_p[c] = pc;
      }
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += ENV_T) {
      pmf_col[(size_t)r * W + c0 + c] = (float)__ddiv_rn(s_w[c], acc);
      put_cdf(cdf_col, cdf_col_lo, (size_t)r * W + c0 + c, __ddiv_rn(s_p[c], acc));
    }
  }
}

__global__ void __launch_bounds__(ENV_T) k_env_marginal(const double* __restrict__ rowsum, int H,
                                                        float* __restrict__ pmf_row, float* __restrict__ cdf_row,
                                                        float* __restrict__ cdf_row_lo) {
  __shared__ double s_pre[ENV_CH];
  __shared__ double s_total;
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int r = 0; r < H; ++r) total = __dadd_rn(total, rowsum[r]);
    s_total = total;
  }
  double pre = 0.0;  // running prefix, held by thread 0
  for (int r0 = 0; r0 < H; r0 += ENV_CH) {
    const int n = min(ENV_CH, H - r0);
    __syncthreads();
    if (threadIdx.x == 0)
      for (int r = 0; r < n; ++r) {
        pre = __dadd_rn(pre, rowsum[r0 + r]);
        s_pre[r] = pre;
      }
    __syncthreads();
    const double total = s_total;
    for (int r = threadIdx.x; r < n; r += ENV_T) {
      pmf_row[r0 + r] = (float)__ddiv_rn(rowsum[r0 + r], total);
      put_cdf(cdf_row, cdf_row_lo, r0 + r, __ddiv_rn(s_pre[r], total));
    }
  }
}

// Instance table of one request: copy each object's current version entry.
__global__ void k_gather_insts(InstPtrs src, Inst* __restrict__ dst, int n) {
  const int k = blockIdx.x;
  if (k >= n) return;
  const float4* s = reinterpret_cast<const float4*>(src.p[k]);
  float4* d = reinterpret_cast<float4*>(dst + k);
  if (threadIdx.x < (int)(sizeof(Inst) / sizeof(float4))) d[threadIdx.x] = s[threadIdx.x];
}

__global__ void k_philox(const uint4* __restrict__ ctr, int n, uint32_t k0, uint32_t k1, uint4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_object_bounds(const SceneDev& s, const int* offsets_dev, int n_obj, int max_obj_n, int* bounds,
                                 cudaStream_t st) {
  k_bounds_init<<<(6 * n_obj + 127) / 128, 128, 0, st>>>(bounds, 6 * n_obj);
  dim3 grid(max(1, min(256, (max_obj_n + 255) / 256)), n_obj);
  k_object_bounds<<<grid, 256, 0, st>>>(s, offsets_dev, bounds);
  return cudaGetLastError();
}

cudaError_t launch_morton(const SceneDev& s, const int* offsets_dev, int n_obj, const int* bounds, unsigned* keys,
                          unsigned* vals, cudaStream_t st) {
  k_morton<<<(s.n + 255) / 256, 256, 0, st>>>(s, offsets_dev, n_obj, bounds, keys, vals);
  return cudaGetLastError();
}

int radix_tiles(int n) { return (n + RS_TILE - 1) / RS_TILE; }

// Sorts (keys, vals) by the 30-bit key, then stably by object of vals.
// Results end in keys/vals; alt buffers are scratch of the same size.
cudaError_t launch_radix_sort(unsigned* keys, unsigned* vals, unsigned* keys_alt, unsigned* vals_alt, int n,
                              const int* offsets_dev, int n_obj, unsigned* counts, cudaStream_t st) {
  const int tiles = radix_tiles(n);
  const int shifts[5] = {0, 8, 16, 24, -1};
  unsigned *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  for (int p = 0; p < 5; ++p) {
    k_radix_hist<<<tiles, RS_THREADS, 0, st>>>(ki, vi, n, shifts[p], offsets_dev, n_obj, counts, tiles);
    k_radix_scan<<<1, 1024, 0, st>>>(counts, 256 * tiles);
    k_radix_scatter<<<tiles, RS_THREADS, 0, st>>>(ki, vi, ko, vo, n, shifts[p], offsets_dev, n_obj, counts,
                                                 tiles);
    unsigned* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  // five passes: the result is in the alternate buffers; copy back
  cudaMemcpyAsync(keys, ki, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(vals, vi, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError();
}

cudaError_t launch_hierarchy(const unsigned* skeys, const int* leaf_off, const int* node_off, int n_obj,
                             int n_nodes_total, float4* nodes, int* leaf_parent, int* node_parent,
                             int2* node_range, cudaStream_t st) {
  if (n_nodes_total > 0)
    k_hierarchy<<<(n_nodes_total + 127) / 128, 128, 0, st>>>(skeys, leaf_off, node_off, n_obj, n_nodes_total,
                                                            nodes, leaf_parent, node_parent, node_range);
  return cudaGetLastError();
}

cudaError_t launch_collapse(const WideArgs& a, cudaStream_t st) {
  if (a.n_objs > 0) k_collapse<<<a.n_objs, COLLAPSE_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_wide_boxes(const WideArgs& a, int n_slots, cudaStream_t st) {
  if (n_slots > 0) k_wide_boxes<<<(n_slots + 255) / 256, 256, 0, st>>>(a, n_slots);
  return cudaGetLastError();
}

cudaError_t launch_pack_fit(const SceneDev& s, const FitArgs& a, cudaStream_t st) {
  if (a.n_leaves > 0) k_pack_fit<<<(a.n_leaves + 127) / 128, 128, 0, st>>>(s, a);
  return cudaGetLastError();
}

cudaError_t launch_rigid(const SceneDev& s, int beg, int end, const Mat34& T, cudaStream_t st) {
  if (end > beg) k_rigid<<<(end - beg + 255) / 256, 256, 0, st>>>(s, beg, end, T);
  return cudaGetLastError();
}

cudaError_t launch_material(const SceneDev& s, int beg, int end, float3 rgb, int set_rgb, float metal, float rough,
                            cudaStream_t st) {
  if (end > beg) k_material<<<(end - beg + 255) / 256, 256, 0, st>>>(s, beg, end, rgb, set_rgb, metal, rough);
  return cudaGetLastError();
}

cudaError_t launch_env_tables(const float* rgb, const double* sin_row, int H, int W, double* rowsum, float* pmf_row,
                              float* cdf_row, float* pmf_col, float* cdf_col, float* cdf_row_lo, float* cdf_col_lo,
                              cudaStream_t st) {
  k_env_rows<<<H, ENV_T, 0, st>>>(rgb, sin_row, H, W, rowsum, pmf_col, cdf_col, cdf_col_lo);
  k_env_marginal<<<1, ENV_T, 0, st>>>(rowsum, H, pmf_row, cdf_row, cdf_row_lo);
  return cudaGetLastError();
}

cudaError_t launch_gather_insts(const InstPtrs& src, Inst* dst, int n, cudaStream_t st) {
  if (n > 0) k_gather_insts<<<n, 32, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, int n, uint32_t k0, uint32_t k1, uint32_t* out, cudaStream_t st) {
  if (n > 0)
    k_philox<<<(n + 127) / 128, 128, 0, st>>>(reinterpret_cast<const uint4*>(ctr), n, k0, k1,
                                             reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

}  // namespace lf
