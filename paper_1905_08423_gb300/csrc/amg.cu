// Levels of an algebraic multigrid hierarchy on the GPU: aggregation and the
// smoothed prolongator, so that the triple products of a whole hierarchy
// (Section 4.2.2: twelve levels, eleven products C = P^T A P) can be formed
// on the device.  The paper takes its coarsening from a cited work; this file
// implements one reading of it (smoothed aggregation):
//
//  * Aggregation by repeated pairwise matching.  In one round every unmatched
//    node picks its strongest unmatched neighbour node; a pair whose members
//    picked each other is matched.  The key of an edge (a, b) is
//    (strength, hash(min(a,b), max(a,b))): it is the same seen from both
//    ends, so the globally strongest edge is always mutual and every round
//    makes progress (locally dominant edges).  Strength between two nodes
//    is the largest |A(i,j)| over their members i, j (a maximum, exact in
//    any order).  Rounds repeat until none matches or `rounds` is reached,
//    then up to `rounds` more rounds key the edges by the hash alone (random
//    priorities, which mop up what long chains of decreasing strength left);
//    a node still unmatched joins the pair with which it has the strongest
//    edge, and stays alone only without a paired neighbour.  Pass k matches
//    the nodes of pass k-1.
//  * Tentative prolongator T(i, agg(i)) = 1 and the smoothed prolongator
//    P = (I - omega D^-1 A_F) T, A_F the diagonal and the strong entries of A
//    (|A(i,j)| >= theta * max_{k != i} |A(i,k)|), D = diag(A):
//    P(i, a) = [agg(i) = a] - omega / A(i,i) * sum over j in A_F(i,:) with
//    agg(j) = a of A(i,j).  Its pattern is the pattern of A_F T, formed by the
//    library's row-wise symbolic product.
#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"

namespace ptap {

int union_pattern_ab(Tracker& mem, const CsrI& A, const CsrI& B, const Config& cfg, int32_t* rp,
                     int32_t** ci, int64_t* nnz, int32_t* status, int* spilled, cudaStream_t s);

namespace {

__host__ __device__ inline uint32_t edge_hash(int32_t a, int32_t b) {
  const uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
  uint32_t h = lo * 0x9E3779B1u ^ (hi + 0x7F4A7C15u + (lo << 6) + (lo >> 2));
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  return h ^ (h >> 16);
}

// (strength, hash) ordering of two candidate edges; true if (w1, h1) > (w2, h2).
__device__ inline bool stronger(double w1, uint32_t h1, double w2, uint32_t h2) {
  return w1 > w2 || (w1 == w2 && h1 > h2);
}

// One round of picks.  Node a (members mem_ptr[a] .. mem_ptr[a+1] of the
// fine rows, listed in members) picks the unmatched node b != a with the
// strongest edge; pick[a] = b, or -1 if it is matched or has no candidate.
// With use_strength false the key is the hash alone (random priorities: the
// rounds that mop up nodes that long chains of decreasing strength left
// unmatched converge fast).
template <typename V>
__global__ void k_pick(CsrV<V> A, const int32_t* __restrict__ node_of, const int32_t* __restrict__ mem_ptr,
                       const int32_t* __restrict__ members, int32_t nnodes, const int32_t* __restrict__ partner,
                       int32_t* __restrict__ pick, bool use_strength) {
  for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < nnodes; a += gridDim.x * blockDim.x) {
    int32_t best = -1;
    double bw = -1.0;
    uint32_t bh = 0;
    if (partner[a] < 0) {
      for (int32_t m = mem_ptr[a]; m < mem_ptr[a + 1]; ++m) {
        const int32_t i = members[m];
        for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
          const int32_t b = node_of[A.ci[e]];
          if (b == a || partner[b] >= 0) continue;
          const double w = use_strength ? fabs((double)A.val[e]) : 0.0;
          const uint32_t h = edge_hash(a, b);
          if (stronger(w, h, bw, bh) || (w == bw && h == bh && b < best)) {
            best = b;
            bw = w;
            bh = h;
          }
        }
      }
    }
    pick[a] = best;
  }
}

// Mutual picks become pairs; counts the matches of this round.
__global__ void k_match(const int32_t* __restrict__ pick, int32_t nnodes, int32_t* __restrict__ partner,
                        int32_t* matched) {
  for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < nnodes; a += gridDim.x * blockDim.x) {
    const int32_t b = pick[a];
    if (b >= 0 && pick[b] == a) {
      partner[a] = b;
      if (a < b) atomicAdd(matched, 1);
    }
  }
}

// A node left unmatched joins the pair with which it has the strongest edge
// (same key as the picks); att[a] = that pair's leader (its smaller node),
// or -1 if it has no matched neighbour (it then stays alone).  Without this a
// node whose neighbours all paired off would stay a singleton level after
// level, and coarsening would stall.
template <typename V>
__global__ void k_attach(CsrV<V> A, const int32_t* __restrict__ node_of, const int32_t* __restrict__ mem_ptr,
                         const int32_t* __restrict__ members, int32_t nnodes, const int32_t* __restrict__ partner,
                         int32_t* __restrict__ att) {
  for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < nnodes; a += gridDim.x * blockDim.x) {
    int32_t best = -1;
    double bw = -1.0;
    uint32_t bh = 0;
    if (partner[a] < 0) {
      for (int32_t m = mem_ptr[a]; m < mem_ptr[a + 1]; ++m) {
        const int32_t i = members[m];
        for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
          const int32_t b = node_of[A.ci[e]];
          if (b == a || partner[b] < 0) continue;
          const double w = fabs((double)A.val[e]);
          const uint32_t h = edge_hash(a, b);
          if (stronger(w, h, bw, bh) || (w == bw && h == bh && b < best)) {
            best = b;
            bw = w;
            bh = h;
          }
        }
      }
    }
    att[a] = best < 0 ? -1 : min(best, partner[best]);
  }
}

__device__ __forceinline__ int32_t leader_of(int32_t a, const int32_t* partner, const int32_t* att) {
  const int32_t b = partner[a];
  return b >= 0 ? min(a, b) : (att[a] >= 0 ? att[a] : a);
}

// New nodes: pair leaders and nodes that stayed alone, in order of old id.
__global__ void k_leaders(const int32_t* __restrict__ partner, const int32_t* __restrict__ att, int32_t nnodes,
                          int32_t* __restrict__ lead) {
  for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < nnodes; a += gridDim.x * blockDim.x)
    lead[a] = leader_of(a, partner, att) == a ? 1 : 0;
}

__global__ void k_relabel(const int32_t* __restrict__ partner, const int32_t* __restrict__ att,
                          const int32_t* __restrict__ lead_pos, int32_t nnodes, int32_t* __restrict__ new_of_old) {
  for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < nnodes; a += gridDim.x * blockDim.x)
    new_of_old[a] = lead_pos[leader_of(a, partner, att)];
}

__global__ void k_map_rows(int32_t n, const int32_t* __restrict__ old_node, const int32_t* __restrict__ new_of_old,
                           int32_t* __restrict__ new_node) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    new_node[i] = new_of_old[old_node[i]];
}

__global__ void k_new_sizes(const int32_t* __restrict__ new_of_old, int32_t nnodes,
                            const int32_t* __restrict__ mem_ptr, int32_t* __restrict__ size) {
  for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < nnodes; a += gridDim.x * blockDim.x)
    atomicAdd(&size[new_of_old[a]], mem_ptr[a + 1] - mem_ptr[a]);
}

// Members of the new nodes (their order inside a node does not matter: the
// picks take a strict maximum).
__global__ void k_new_members(const int32_t* __restrict__ new_of_old, int32_t nnodes,
                              const int32_t* __restrict__ mem_ptr, const int32_t* __restrict__ members,
                              int32_t* __restrict__ cursor, int32_t* __restrict__ new_members) {
  for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < nnodes; a += gridDim.x * blockDim.x) {
    const int32_t cnt = mem_ptr[a + 1] - mem_ptr[a];
    int32_t o = atomicAdd(&cursor[new_of_old[a]], cnt);
    for (int32_t m = mem_ptr[a]; m < mem_ptr[a + 1]; ++m) new_members[o++] = members[m];
  }
}

__global__ void k_iota(int32_t n, int32_t* __restrict__ x) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) x[i] = i;
}

__global__ void k_one_per_row(int32_t n, int32_t* __restrict__ rp) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) rp[i] = i;
}

// Strength of the entries of A: mask[e] = 1 for an off-diagonal entry with
// |A(i,j)| >= theta * max_{k != i} |A(i,k)| (theta = 0: every off-diagonal
// entry), 0 for the diagonal and for weak entries.  Settled once, at
// symbolic time, so the prolongator's pattern does not move with the values.
template <typename V>
__global__ void k_strong(CsrV<V> A, double theta, uint8_t* __restrict__ mask, int32_t* __restrict__ cnt) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nrows; i += gridDim.x * blockDim.x) {
    double mx = 0.0;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
      if (A.ci[e] != i) mx = fmax(mx, fabs((double)A.val[e]));
    const double thr = theta * mx;
    int32_t c = 1;  // the diagonal position of the filtered row
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
      const bool st = A.ci[e] != i && fabs((double)A.val[e]) >= thr;
      mask[e] = st ? 1 : 0;
      c += st ? 1 : 0;
    }
    cnt[i] = c;
  }
}

// Pattern of the filtered operator: the diagonal and the strong entries.
__global__ void k_filtered_fill(CsrI A, const uint8_t* __restrict__ mask, const int32_t* __restrict__ frp,
                                int32_t* __restrict__ fci) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nrows; i += gridDim.x * blockDim.x) {
    int32_t o = frp[i];
    fci[o++] = i;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
      if (mask[e]) fci[o++] = A.ci[e];
  }
}

// Values of P = (I - omega D^-1 A_F) T on its sorted pattern, one thread a
// row: A_F keeps the diagonal and the strong entries of A, D = diag(A).  The
// weak entries are dropped, not lumped into the diagonal: on coarse levels,
// whose off-diagonal entries take both signs, lumping can cancel most of the
// diagonal and blow P's entries up.
template <typename V>
__global__ void k_prolong_values(CsrV<V> A, const uint8_t* __restrict__ mask, const int32_t* __restrict__ agg,
                                 const int32_t* __restrict__ prp, const int32_t* __restrict__ pci, double omega,
                                 V* __restrict__ pval, int32_t* status) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nrows; i += gridDim.x * blockDim.x) {
    const int32_t p0 = prp[i], p1 = prp[i + 1];
    V d = V(0);
    bool has_diag = false;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e)
      if (A.ci[e] == i) {
        has_diag = true;
        d = A.val[e];
      }
    for (int32_t q = p0; q < p1; ++q) pval[q] = V(0);
    auto pos = [&](int32_t a) {
      int32_t lo = p0, hi = p1;
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (pci[mid] < a) lo = mid + 1;
        else hi = mid;
      }
      return (lo < p1 && pci[lo] == a) ? lo : -1;
    };
    const int32_t own = pos(agg[i]);
    if (own < 0 || !has_diag || d == V(0)) {
      atomicExch(status, PTAP_ERR_INVALID);  // no diagonal entry, or the pattern is not this P's
      continue;
    }
    pval[own] = V(1) - (V)omega;   // the diagonal's own term: 1 - omega d / d
    const V f = (V)(omega) / d;
    for (int32_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
      if (!mask[e]) continue;
      const int32_t q = pos(agg[A.ci[e]]);
      if (q < 0) {
        atomicExch(status, PTAP_ERR_PATTERN);
        continue;
      }
      pval[q] -= f * A.val[e];
    }
  }
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), num_sms() * 8)); }

}  // namespace
}  // namespace ptap

struct ptap_prolongator {
  ptap::Tracker mem;
  cudaStream_t stream = nullptr;
  int32_t n = 0, m = 0;
  int64_t nnz_a = 0, nnz = 0;
  int32_t* agg = nullptr;  // copy of the aggregate of every fine row
  uint8_t* mask = nullptr; // strong entries of A (settled at symbolic time)
  int32_t* rp = nullptr;
  int32_t* ci = nullptr;
  int32_t* status = nullptr;
};

namespace ptap {
namespace {

template <typename V>
int aggregate_t(const ptap_csr* Ain, int32_t passes, int32_t rounds, int32_t* agg, int32_t* n_agg,
                Tracker& mem, cudaStream_t s) {
  const int32_t n = Ain->nrows;
  CsrV<V> A{Ain->nrows, Ain->ncols, Ain->row_ptr, Ain->col_idx, (const V*)Ain->val};
  Scratch sc(&mem);
  int32_t *node_of = nullptr, *mem_ptr = nullptr, *members = nullptr, *partner = nullptr, *pick = nullptr,
          *counter = nullptr, *lead = nullptr, *lead_pos = nullptr, *new_of_old = nullptr, *size = nullptr,
          *new_ptr = nullptr, *new_members = nullptr, *att = nullptr;
  PTAP_TRY(sc.get(&node_of, std::max(n, 1)));
  PTAP_TRY(sc.get(&mem_ptr, (int64_t)n + 1));
  PTAP_TRY(sc.get(&members, std::max(n, 1)));
  PTAP_TRY(sc.get(&partner, std::max(n, 1)));
  PTAP_TRY(sc.get(&pick, std::max(n, 1)));
  PTAP_TRY(sc.get(&counter, 1));
  PTAP_TRY(sc.get(&lead, (int64_t)n + 1));
  PTAP_TRY(sc.get(&lead_pos, (int64_t)n + 1));
  PTAP_TRY(sc.get(&new_of_old, std::max(n, 1)));
  PTAP_TRY(sc.get(&size, (int64_t)n + 1));
  PTAP_TRY(sc.get(&new_ptr, (int64_t)n + 1));
  PTAP_TRY(sc.get(&new_members, std::max(n, 1)));
  PTAP_TRY(sc.get(&att, (int64_t)n + 1));  // attachments, then the member cursor of each new node
  // pass 0 nodes: the fine rows themselves
  k_iota<<<grid_of(n + 1), 256, 0, s>>>(n, mem_ptr);
  k_iota<<<grid_of(n), 256, 0, s>>>(n - 1, members);
  k_iota<<<grid_of(n), 256, 0, s>>>(n - 1, node_of);
  PTAP_LAUNCHED();
  int32_t nnodes = n;
  for (int32_t pass = 0; pass < passes && nnodes > 1; ++pass) {
    PTAP_CUDA(cudaMemsetAsync(partner, 0xff, (size_t)nnodes * sizeof(int32_t), s));
    // `rounds` rounds keyed by strength, then up to `rounds` keyed by the hash
    // alone; a round that matches nothing ends its phase
    for (int32_t r = 0; r < 2 * rounds; ++r) {
      const bool strength = r < rounds;
      PTAP_CUDA(cudaMemsetAsync(counter, 0, sizeof(int32_t), s));
      k_pick<V><<<grid_of(nnodes), 256, 0, s>>>(A, node_of, mem_ptr, members, nnodes, partner, pick, strength);
      k_match<<<grid_of(nnodes), 256, 0, s>>>(pick, nnodes, partner, counter);
      PTAP_LAUNCHED();
      int32_t matched = 0;
      PTAP_CUDA(cudaMemcpyAsync(&matched, counter, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      PTAP_CUDA(cudaStreamSynchronize(s));
      if (matched == 0) {
        if (!strength) break;
        r = rounds - 1;  // on to the hash-keyed rounds
      }
    }
    // unmatched nodes join their strongest neighbouring pair; new nodes are
    // the pair leaders and the nodes left alone, in order of their old id
    k_attach<V><<<grid_of(nnodes), 256, 0, s>>>(A, node_of, mem_ptr, members, nnodes, partner, att);
    k_leaders<<<grid_of(nnodes), 256, 0, s>>>(partner, att, nnodes, lead);
    PTAP_LAUNCHED();
    int64_t nnew = 0;
    PTAP_TRY(exclusive_scan(mem, lead, lead_pos, nnodes, &nnew, s));
    k_relabel<<<grid_of(nnodes), 256, 0, s>>>(partner, att, lead_pos, nnodes, new_of_old);
    k_map_rows<<<grid_of(n), 256, 0, s>>>(n, node_of, new_of_old, node_of);
    PTAP_CUDA(cudaMemsetAsync(size, 0, (size_t)(nnew + 1) * sizeof(int32_t), s));
    k_new_sizes<<<grid_of(nnodes), 256, 0, s>>>(new_of_old, nnodes, mem_ptr, size);
    PTAP_LAUNCHED();
    PTAP_TRY(exclusive_scan(mem, size, new_ptr, nnew, nullptr, s));
    PTAP_CUDA(cudaMemcpyAsync(att, new_ptr, (size_t)nnew * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    k_new_members<<<grid_of(nnodes), 256, 0, s>>>(new_of_old, nnodes, mem_ptr, members, att, new_members);
    PTAP_LAUNCHED();
    std::swap(mem_ptr, new_ptr);
    std::swap(members, new_members);
    nnodes = (int32_t)nnew;
  }
  PTAP_CUDA(cudaMemcpyAsync(agg, node_of, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  *n_agg = nnodes;
  return PTAP_OK;
}

}  // namespace
}  // namespace ptap

extern "C" int ptap_aggregate(const ptap_csr* A, int32_t passes, int32_t rounds, int32_t* agg, int32_t* n_agg,
                              const ptap_allocator* alloc, void* stream) {
  ptap::Range range("ptap_aggregate");
  if (!A || !agg || !n_agg || passes < 0 || passes > 8 || rounds < 1) return PTAP_ERR_INVALID;
  PTAP_TRY(ptap::check_csr_host(A, true));
  if (A->nrows != A->ncols) return PTAP_ERR_INVALID;
  if (A->nrows == 0) {
    *n_agg = 0;
    return PTAP_OK;
  }
  ptap::Tracker mem;
  mem.init(alloc, (cudaStream_t)stream);
  const int rc = A->dtype == PTAP_F64
                     ? ptap::aggregate_t<double>(A, passes, rounds, agg, n_agg, mem, (cudaStream_t)stream)
                     : ptap::aggregate_t<float>(A, passes, rounds, agg, n_agg, mem, (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  mem.release_all();
  return rc;
}

extern "C" int ptap_prolongator_symbolic(const ptap_csr* A, const int32_t* agg, int32_t n_agg, double theta,
                                         const ptap_allocator* alloc, void* stream, ptap_prolongator** out) {
  using namespace ptap;
  Range range("ptap_prolongator_symbolic");
  if (!A || !agg || !out || n_agg < 0) return PTAP_ERR_INVALID;
  *out = nullptr;
  PTAP_TRY(check_csr_host(A, true));  // the strength of connection reads A's values
  if (A->nrows != A->ncols || (A->nrows > 0 && n_agg < 1) || !(theta >= 0.0 && theta <= 1.0))
    return PTAP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  ptap_prolongator* p = new (std::nothrow) ptap_prolongator();
  if (!p) return PTAP_ERR_OOM;
  p->mem.init(alloc, s);
  p->stream = s;
  p->n = A->nrows;
  p->m = n_agg;
  p->nnz_a = A->nnz;
  auto body = [&]() -> int {
    PTAP_TRY(p->mem.get_n(&p->status, 1));
    PTAP_CUDA(cudaMemsetAsync(p->status, 0, sizeof(int32_t), s));
    PTAP_TRY(p->mem.get_n(&p->agg, std::max(p->n, 1)));
    PTAP_TRY(p->mem.get_n(&p->rp, (int64_t)p->n + 1));
    if (p->n > 0)
      PTAP_CUDA(cudaMemcpyAsync(p->agg, agg, (size_t)p->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    // strong entries, the filtered operator's pattern, then the pattern of
    // A_F T (T the tentative prolongator: one entry a row)
    Scratch sc(&p->mem);
    int32_t *trp = nullptr, *fcnt = nullptr, *frp = nullptr, *fci = nullptr;
    PTAP_TRY(p->mem.get_n(&p->mask, std::max<int64_t>(p->nnz_a, 1)));
    PTAP_TRY(sc.get(&trp, (int64_t)p->n + 1));
    PTAP_TRY(sc.get(&fcnt, (int64_t)p->n + 1));
    PTAP_TRY(sc.get(&frp, (int64_t)p->n + 1));
    k_one_per_row<<<grid_of(p->n + 1), 256, 0, s>>>(p->n, trp);
    if (A->dtype == PTAP_F64)
      k_strong<double><<<grid_of(p->n), 256, 0, s>>>(
          CsrV<double>{A->nrows, A->ncols, A->row_ptr, A->col_idx, (const double*)A->val}, theta, p->mask, fcnt);
    else
      k_strong<float><<<grid_of(p->n), 256, 0, s>>>(
          CsrV<float>{A->nrows, A->ncols, A->row_ptr, A->col_idx, (const float*)A->val}, theta, p->mask, fcnt);
    PTAP_LAUNCHED();
    int64_t fnnz = 0;
    PTAP_TRY(exclusive_scan(p->mem, fcnt, frp, p->n, &fnnz, s));
    PTAP_TRY(sc.get(&fci, std::max<int64_t>(fnnz, 1)));
    k_filtered_fill<<<grid_of(p->n), 256, 0, s>>>(CsrI{A->nrows, A->ncols, A->row_ptr, A->col_idx}, p->mask,
                                                   frp, fci);
    PTAP_LAUNCHED();
    CsrI Ai{A->nrows, A->ncols, frp, fci};
    CsrI Ti{p->n, n_agg, trp, p->agg};
    Config cfg;
    int spilled = 0;
    PTAP_TRY(union_pattern_ab(p->mem, Ai, Ti, cfg, p->rp, &p->ci, &p->nnz, p->status, &spilled, s));
    PTAP_CUDA(cudaStreamSynchronize(s));
    int32_t st = 0;
    PTAP_CUDA(cudaMemcpy(&st, p->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    return st;
  };
  const int rc = body();
  if (rc != PTAP_OK) {
    cudaStreamSynchronize(s);
    p->mem.release_all();
    delete p;
    return rc;
  }
  *out = p;
  return PTAP_OK;
}

extern "C" int ptap_prolongator_pattern(const ptap_prolongator* p, int32_t* nrows, int32_t* ncols, int64_t* nnz,
                                        const int32_t** row_ptr, const int32_t** col_idx) {
  if (!p) return PTAP_ERR_INVALID;
  if (nrows) *nrows = p->n;
  if (ncols) *ncols = p->m;
  if (nnz) *nnz = p->nnz;
  if (row_ptr) *row_ptr = p->rp;
  if (col_idx) *col_idx = p->ci;
  return PTAP_OK;
}

extern "C" int ptap_prolongator_numeric(ptap_prolongator* p, const ptap_csr* A, double omega, void* P_val,
                                        void* stream) {
  using namespace ptap;
  Range range("ptap_prolongator_numeric");
  if (!p || !A) return PTAP_ERR_INVALID;
  PTAP_TRY(check_csr_host(A, true));
  if (A->nrows != p->n || A->ncols != p->n || A->nnz != p->nnz_a) return PTAP_ERR_PATTERN;
  if (p->nnz > 0 && !P_val) return PTAP_ERR_INVALID;
  if (p->n == 0) return PTAP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (A->dtype == PTAP_F64)
    k_prolong_values<double><<<grid_of(p->n), 256, 0, s>>>(
        CsrV<double>{A->nrows, A->ncols, A->row_ptr, A->col_idx, (const double*)A->val}, p->mask, p->agg, p->rp,
        p->ci, omega, (double*)P_val, p->status);
  else
    k_prolong_values<float><<<grid_of(p->n), 256, 0, s>>>(
        CsrV<float>{A->nrows, A->ncols, A->row_ptr, A->col_idx, (const float*)A->val}, p->mask, p->agg, p->rp,
        p->ci, omega, (float*)P_val, p->status);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

extern "C" int ptap_prolongator_check(ptap_prolongator* p, void* stream) {
  if (!p) return PTAP_ERR_INVALID;
  int32_t st = 0;
  PTAP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  PTAP_CUDA(cudaMemcpy(&st, p->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (st) PTAP_CUDA(cudaMemset(p->status, 0, sizeof(int32_t)));
  return st;
}

extern "C" void ptap_prolongator_destroy(ptap_prolongator* p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  p->mem.release_all();
  delete p;
}
