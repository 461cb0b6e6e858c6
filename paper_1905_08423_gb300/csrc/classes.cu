// Fine-row structure classes for the fast numeric path (symbolic phase).
//
// The numeric product is repeated on a fixed symbolic result (Section 4.1:
// one symbolic, eleven numeric; Section 4.2, Table 8: caching intermediate
// data).  For a fine row I, everything the numeric phase does except reading
// values is fixed by the patterns: which P rows the row of A P combines
// (Alg. 3), which distinct columns that row has, and where each product
// P(I,i) (A P)(I,j) lands in row i of the preallocated C (Alg. 8).  This file
// computes that description -- the row's "signature" -- for every fine row,
// and deduplicates identical signatures into classes.  Operators discretised
// on meshes have few classes (hundreds), so the numeric kernel can run 32
// fine rows of one class in lockstep from one small program, with no hashing
// and no searching.
//
// Signature ("program") of fine row I, in the layout the kernel reads:
//   [0] na  entries of A(I,:)  (<= kFastMaxA)     [1] r  distinct columns of (A P)(I,:) (<= kFastMaxR)
//   [2] pI  entries of P(I,:)  (<= kFastMaxP)     [3..8) zero
//   [8 .. 8+A8)      p_a = entries of P(k_a,:), k_a the a-th column of A(I,:); A8 = na rounded up to 8
//   [.. +8*na)       t(a,b) at a*8+b: slot of P(k_a,:)'s b-th column in the sorted row of A P
//   [.. +8*r)        sigma at t*8+s: position of the t-th column in C row P(I,:)'s s-th column
// All padding bytes are zero, so equal rows have byte-equal programs.
// Rows outside these limits (or with C rows longer than 255) make the plan
// fall back to the general kernel.
//
// Deduplication: a 64-bit hash of each signature goes into an open-addressing
// table (atomicCAS); the row that inserts a hash writes its signature to the
// program pool and flags it ready; every other row compares its own signature
// byte by byte with the pool entry of its hash -- at once when the entry is
// ready, otherwise in a short second pass -- so a hash collision can only
// demote rows to the general path, never corrupt results.  No warp waits on
// another.  In front of it sits a table of row shapes (the patterns a
// program depends on, relative to the row's first coarse column): a row
// whose shape was seen takes that shape's class without computing its
// program (k_class_build).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace ptap {

namespace {

constexpr unsigned long long kEmptyKey = ~0ull;

struct SigGeom {
  CsrI A, P, C;
};

// Warp-cooperative signature of fine row I into sig[] (shared memory);
// returns its length, or -1 if the row is outside the fast-path limits.
// cand/keys: kFastMaxT ints of shared memory each.
//
// Rows with at most 32 products stay in registers: the products' columns are
// sorted with their positions as 64-bit keys by a warp bitonic sort, so each
// product learns its slot in the sorted row of A P from a ballot.  Longer
// rows take a shared-memory bitonic sort and binary searches.
__device__ int compute_sig(const SigGeom& g, int32_t I, uint8_t* sig, int32_t* cand, int32_t* keys,
                           int32_t* status) {
  const int lane = threadIdx.x & 31;
  const int32_t a0 = g.A.rp[I], na = g.A.rp[I + 1] - a0;
  const int32_t p0 = g.P.rp[I], pI = g.P.rp[I + 1] - p0;
  if (na > kFastMaxA || pI > kFastMaxP || pI <= 0) return -1;
  int32_t pb = 0, pa = 0;
  if (lane < na) {
    const int32_t k = g.A.ci[a0 + lane];
    pb = g.P.rp[k];
    pa = g.P.rp[k + 1] - pb;
  }
  if (__any_sync(0xffffffffu, pa > kFastMaxB)) return -1;
  int32_t off = pa;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, off, d);
    if (lane >= d) off += y;
  }
  const int32_t T = __shfl_sync(0xffffffffu, off, 31);
  off -= pa;
  for (int32_t b = 0; b < pa; ++b) cand[off + b] = g.P.ci[pb + b];
  // zero the whole program region first (padding must be deterministic)
  for (int x = lane; x < kFastSigCap / 4; x += 32) reinterpret_cast<uint32_t*>(sig)[x] = 0u;
  __syncwarp();
  int32_t r = 0;
  const bool small = T <= 32;
  if (small) {
    // sort (column, position) pairs; then slots by ranking the first occurrences
    unsigned long long v = lane < T ? ((unsigned long long)(uint32_t)cand[lane] << 32) | (unsigned)lane : ~0ull;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, j);
        const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
        v = keep_min ? (u < v ? u : v) : (u > v ? u : v);
      }
    const int32_t key = (int32_t)(v >> 32);
    const int32_t up = __shfl_up_sync(0xffffffffu, key, 1);
    const bool first = lane < T && (lane == 0 || up != key);
    const unsigned m = __ballot_sync(0xffffffffu, first);
    const unsigned le = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    const int32_t t = __popc(m & le) - 1;
    r = __popc(m);
    __syncwarp();
    if (first) keys[t] = key;
    if (lane < T) cand[(int32_t)(v & 0xffffffffu)] = t;  // cand now holds each product's slot
    __syncwarp();
  } else {
    for (int32_t x = lane; x < T; x += 32) keys[x] = cand[x];
    __syncwarp();
    // ascending sort of keys[0, T) (bitonic, comparators all ascending;
    // sizes and strides are powers of two, so shifts and masks index them)
    int p = 1, lp = 0;
    while (p < T) {
      p <<= 1;
      ++lp;
    }
    for (int ls = 1; ls <= lp; ++ls)
      for (int lj = ls - 1; lj >= 0; --lj) {
        const int size = 1 << ls, j = 1 << lj;
        for (int t = lane; t < (p >> 1); t += 32) {
          const int hi = t >> lj, lo = t & (j - 1);
          int x, y;
          if (lj == ls - 1) {
            x = hi * size + lo;
            y = hi * size + size - 1 - lo;
          } else {
            x = (hi << (lj + 1)) + lo;
            y = x + j;
          }
          if (y < T) {
            const int32_t kx = keys[x], ky = keys[y];
            if (kx > ky) {
              keys[x] = ky;
              keys[y] = kx;
            }
          }
        }
        __syncwarp();
      }
    // unique, in place (each 32-wide window is read before it is written)
    int32_t prev = 0;
    for (int32_t base = 0; base < T; base += 32) {
      const int32_t x = base + lane;
      const int32_t kx = x < T ? keys[x] : 0;
      int32_t up = __shfl_up_sync(0xffffffffu, kx, 1);
      if (lane == 0) up = prev;
      const bool first = x < T && (x == 0 || up != kx);
      const unsigned m = __ballot_sync(0xffffffffu, first);
      prev = __shfl_sync(0xffffffffu, kx, 31);
      __syncwarp();
      if (first) keys[r + __popc(m & ((1u << lane) - 1u))] = kx;
      r += __popc(m);
      __syncwarp();
    }
  }
  if (r > kFastMaxR) return -1;
  // slot of each of this lane's products (lane = a, up to kFastMaxB of them)
  const int A8 = (na + 7) & ~7;
  const int tsec = 8 + A8;
  if (lane < na) {
    sig[8 + lane] = (uint8_t)pa;
    for (int32_t b = 0; b < pa; ++b) {
      int32_t lo;
      if (small) {
        lo = cand[off + b];
      } else {
        const int32_t key = cand[off + b];
        int32_t hi = r;
        lo = 0;
        while (lo < hi) {
          const int32_t mid = (lo + hi) >> 1;
          if (keys[mid] < key) lo = mid + 1;
          else hi = mid;
        }
      }
      sig[tsec + lane * 8 + b] = (uint8_t)lo;
    }
  }
  const int ssec = tsec + 8 * na;
  const int tcur = ssec + 8 * r;
  // positions in the rows of C (sigma): every (s, t) pair searches its C row
  // in parallel (the rows are short and shared by neighbouring fine rows, so
  // the searches mostly hit L1)
  bool too_long = false;
  for (int32_t e = lane; e < pI * r; e += 32) {
    const int32_t s = e / r, t = e - s * r;
    const int32_t i = g.P.ci[p0 + s];
    const int32_t c0 = g.C.rp[i], L = g.C.rp[i + 1] - c0;
    if (L > 255) {
      too_long = true;
      continue;
    }
    const int32_t kt = keys[t];
    int32_t lo = 0, hi = L;
    while (lo < hi) {
      const int32_t mid = (lo + hi) >> 1;
      if (g.C.ci[c0 + mid] < kt) lo = mid + 1;
      else hi = mid;
    }
    if (lo >= L || g.C.ci[c0 + lo] != kt) atomicExch(status, PTAP_ERR_PATTERN);
    sig[ssec + t * 8 + s] = (uint8_t)lo;
  }
  if (__any_sync(0xffffffffu, too_long)) return -1;
  if (lane == 0) {
    sig[0] = (uint8_t)na;
    sig[1] = (uint8_t)r;
    sig[2] = (uint8_t)pI;
  }
  __syncwarp();
  return tcur;
}

// Length of a program from its header (host and device).
__host__ __device__ inline int program_length(const uint8_t* g) {
  return 8 + ((g[0] + 7) & ~7) + 8 * g[0] + 8 * g[1];
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Order-sensitive 64-bit hash of sig[0, len), warp-cooperative.
__device__ unsigned long long sig_hash(const uint8_t* sig, int len) {
  const int lane = threadIdx.x & 31;
  unsigned long long h = 0xcbf29ce484222325ull ^ mix64((unsigned long long)(lane + 1) * 0x9e3779b97f4a7c15ull);
  const uint32_t* w = reinterpret_cast<const uint32_t*>(sig);  // len is a multiple of 8
  for (int x = lane; x < (len >> 2); x += 32) h = (h ^ (unsigned long long)w[x]) * 0x100000001b3ull;
  h = mix64(h + (unsigned long long)lane * 0x632be59bd9b4e019ull + (unsigned long long)len);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, d);
  return h == kEmptyKey ? 0 : h;
}

struct ClassArgs {
  SigGeom g;
  int32_t n;
  unsigned long long* tkey;  // table keys (hash), kEmptyKey = free
  int32_t* tready;           // per slot: 1 once the key's program is in the pool
  int32_t* tcls;             // class id per slot
  int tlog2;
  uint8_t* pool;
  int64_t pool_cap;
  int32_t* class_off;        // [K+1] pool offset per class (class_off[k] = start)
  int32_t* counters;         // [0] classes, [1] pool bytes used, [2] slow rows, [3] overflow,
                             // [4] rows left to verify, [5] shape pool words used
  int32_t* row_class;        // per fine row: class id, or -1 (no P entries), or -2 (general
                             // path), or -3 (to be verified by k_class_verify)
  int32_t* status;
  // the shape table (see k_class_build): keys, ready flags, class of each
  // shape, and the shape pool (int32 words); counters[5] counts pool words
  unsigned long long* skey;
  int32_t* sready;
  int32_t* scls;
  int32_t* spool;
  int32_t* soff;             // pool offset of each slot's shape
  int64_t spool_cap;
  const int32_t* crep;       // representative of each C row (k_crow_rep), -1 for rows over 255
  int32_t* vlist;            // the rows marked -3, in the order they were met (first vcap of them)
  int32_t vcap;
};

constexpr int kSigWarps = 4;
constexpr uint32_t kMaxProbes = 256;  // linear probes of the class table before it counts as full

constexpr int kShapeCap = 320;       // words of a row's shape kept on chip; longer rows skip the shape table

struct SigSmem {
  __align__(16) uint8_t sig[kSigWarps][kFastSigCap];
  int32_t cand[kSigWarps][kFastMaxT];
  int32_t keys[kSigWarps][kFastMaxT];
  int32_t shape[kSigWarps][3][kShapeCap];  // per warp: the row's shape and two remembered ones
};

// The shape of fine row I: everything its program depends on, relative to
// c = the first column of P(I,:):
//   na, pI, (P.ci of P(I,:)) - c, then per entry a of A(I,:): pa, (columns of
//   P(k_a,:)) - c, then per entry s of P(I,:): the representative of C row
//   i_s (k_crow_rep: equal representatives, equal columns relative to i_s).
// Two rows with equal shapes have equal programs: the slots of A P follow
// from the order of the relative columns, the positions in C from the
// relative C rows.  Returns the length in words; -1 if the row is outside
// the fast-path limits (as compute_sig would find, except the row of A P
// being too long, which its program reveals); -4 if the shape exceeds the
// on-chip buffer.
__device__ int compute_shape(const SigGeom& g, const int32_t* __restrict__ crep, int32_t I, int32_t* sh) {
  const int lane = threadIdx.x & 31;
  const int32_t a0 = g.A.rp[I], na = g.A.rp[I + 1] - a0;
  const int32_t p0 = g.P.rp[I], pI = g.P.rp[I + 1] - p0;
  if (na > kFastMaxA || pI > kFastMaxP || pI <= 0) return -1;
  const int32_t base = g.P.ci[p0];
  int32_t pb = 0, pa = 0;
  if (lane < na) {
    const int32_t k = g.A.ci[a0 + lane];
    pb = g.P.rp[k];
    pa = g.P.rp[k + 1] - pb;
  }
  if (__any_sync(0xffffffffu, pa > kFastMaxB)) return -1;
  int32_t off = lane < na ? 1 + pa : 0;  // inclusive scan of 1 + pa over the entries of A(I,:)
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, off, d);
    if (lane >= d) off += y;
  }
  const int32_t asec = __shfl_sync(0xffffffffu, off, 31);  // words of the A section
  int len = 2 + pI + asec;
  if (len > kShapeCap) return -4;
  if (lane == 0) {
    sh[0] = na;
    sh[1] = pI;
  }
  if (lane < pI) sh[2 + lane] = g.P.ci[p0 + lane] - base;
  if (lane < na) {
    int32_t o = 2 + pI + off - (1 + pa);
    sh[o] = pa;
    for (int32_t b = 0; b < pa; ++b) sh[o + 1 + b] = g.P.ci[pb + b] - base;
  }
  // the C rows of P(I,:): their representatives (rows with equal columns
  // relative to their own index share one, see k_crow_rep); with the
  // section of P(I,:) above, which fixes each i_s - c, this fixes the C rows
  // relative to c
  int32_t rep = 0;
  if (lane < pI) rep = crep[g.P.ci[p0 + lane]];
  if (__any_sync(0xffffffffu, lane < pI && rep < 0)) return -1;  // a C row too long for a program
  if (lane < pI) sh[len + lane] = rep;
  len += pI;
  __syncwarp();
  return len;
}

// Order-sensitive 64-bit hash of the words w[0, len), warp-cooperative.
__device__ unsigned long long words_hash(const int32_t* w, int len);


// Byte-compares the warp's signature sig[0, len) with the pool entry of class
// cls; reads bypass L1 (entries may have been written by another SM during
// this launch).
__device__ bool same_program(const ClassArgs& c, int32_t cls, const uint8_t* sig, int len) {
  const int lane = threadIdx.x & 31;
  const uint8_t* ref = c.pool + __ldcg(&c.class_off[cls]);
  const int rlen = 8 + ((__ldcg(ref) + 7) & ~7) + 8 * __ldcg(ref) + 8 * __ldcg(ref + 1);
  bool same = rlen == len;
  if (same)
    for (int x = lane; x < len; x += 32) same &= (__ldcg(ref + x) == sig[x]);
  return __all_sync(0xffffffffu, same);
}

__device__ unsigned long long words_hash(const int32_t* w, int len) {
  const int lane = threadIdx.x & 31;
  unsigned long long h = 0x84222325cbf29ce4ull ^ mix64((unsigned long long)(lane + 1) * 0x9e3779b97f4a7c15ull);
  for (int x = lane; x < len; x += 32) h = (h ^ (unsigned long long)(uint32_t)w[x]) * 0x100000001b3ull;
  h = mix64(h + (unsigned long long)lane * 0x632be59bd9b4e019ull + (unsigned long long)len);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, d);
  return h == kEmptyKey ? 0 : h;
}

// Class of the program sig[0, len) in the program table: the row that
// inserts a key publishes its program to the pool and then sets the slot's
// ready flag; a row that finds its key ready compares its program with the
// published bytes.  Returns the class id, -2 (table or pool full, or a hash
// collision: the general path) or -3 (the key's program not yet published;
// k_class_verify settles the row after this launch).  No warp waits.
__device__ int32_t program_class(const ClassArgs& c, const uint8_t* sig, int len) {
  const int lane = threadIdx.x & 31;
  const uint32_t mask = (1u << c.tlog2) - 1u;
  const unsigned long long h = sig_hash(sig, len);
  int role = 0;  // 1: this row publishes the key, 2: the key exists, 0: table full
  uint32_t slot = (uint32_t)(h >> 20) & mask;
  if (lane == 0) {
    // bounded probing: a table this crowded means far too many classes
    for (uint32_t probe = 0; probe <= mask && probe < kMaxProbes; ++probe) {
      unsigned long long old = *(volatile unsigned long long*)&c.tkey[slot];
      if (old == kEmptyKey) old = atomicCAS(&c.tkey[slot], kEmptyKey, h);
      if (old == kEmptyKey) {
        role = 1;
        break;
      }
      if (old == h) {
        role = 2;
        break;
      }
      slot = (slot + 1) & mask;
    }
    if (role == 0) atomicExch(&c.counters[3], 1);
  }
  role = __shfl_sync(0xffffffffu, role, 0);
  slot = __shfl_sync(0xffffffffu, slot, 0);
  int32_t cls = -2;
  if (role == 1) {
    int32_t off = 0;
    if (lane == 0) {
      off = atomicAdd(&c.counters[1], len);
      if ((int64_t)off + len <= c.pool_cap) {
        cls = atomicAdd(&c.counters[0], 1);
        c.class_off[cls] = off;
      } else {
        cls = -1;
        atomicExch(&c.counters[3], 1);
      }
    }
    cls = __shfl_sync(0xffffffffu, cls, 0);
    off = __shfl_sync(0xffffffffu, off, 0);
    if (cls >= 0)
      for (int x = lane; x < len; x += 32) c.pool[off + x] = sig[x];
    __syncwarp();
    if (lane == 0) {
      c.tcls[slot] = cls;
      __threadfence();  // the program and its class id before the flag
      atomicExch(&c.tready[slot], 1);
    }
    if (cls < 0) cls = -2;
  } else if (role == 2) {
    int ready = 0;
    if (lane == 0) ready = atomicAdd(&c.tready[slot], 0);
    ready = __shfl_sync(0xffffffffu, ready, 0);
    __threadfence();
    if (ready) {
      const int32_t k = __ldcg(&c.tcls[slot]);
      cls = (k >= 0 && same_program(c, k, sig, len)) ? k : -2;
    } else {
      cls = -3;
    }
  }
  return cls;
}

// The class of a row from its program (the full path).
__device__ int32_t row_program_class(const ClassArgs& c, int32_t I, SigSmem& sm, int w) {
  const int len = compute_sig(c.g, I, sm.sig[w], sm.cand[w], sm.keys[w], c.status);
  return len < 0 ? -2 : program_class(c, sm.sig[w], len);
}

// Representatives of the rows of C: rep[i] = the first row met, in this
// launch, whose columns relative to its own index equal row i's (C(i,:) - i);
// -1 for a row longer than 255 (outside the class programs).  Equal
// representatives mean equal relative rows, which is all the fine rows'
// programs need of C.  A table keyed by a hash of the relative row holds the
// published representatives; a row compares itself with the representative's
// row (in C itself) before taking it, so a collision only costs a row its
// own representative.  Warps take runs of 32 consecutive rows and remember
// their last two representatives on chip.  No warp waits on another.
struct CrowArgs {
  CsrI C;
  unsigned long long* key;
  int32_t* ready;
  int32_t* rep_of_slot;
  int tlog2;
  int32_t* rep;
};

__device__ bool same_crow(const CsrI& C, int32_t i, int32_t r) {
  const int lane = threadIdx.x & 31;
  const int32_t ci0 = C.rp[i], L = C.rp[i + 1] - ci0, cr0 = C.rp[r];
  if (C.rp[r + 1] - cr0 != L) return false;  // the same in every lane
  bool same = true;
  for (int32_t j = lane; j < L; j += 32) same = same && (C.ci[ci0 + j] - i == C.ci[cr0 + j] - r);
  return __all_sync(0xffffffffu, same);
}

__global__ void __launch_bounds__(128) k_crow_rep(CrowArgs a) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t mask = (1u << a.tlog2) - 1u;
  int32_t memo[2] = {-1, -1};
  unsigned long long memo_h[2] = {kEmptyKey, kEmptyKey};
  const int64_t warps = (int64_t)gridDim.x * 4;
  for (int64_t run = (int64_t)blockIdx.x * 4 + w; run * 32 < a.C.nrows; run += warps) {
    const int64_t i1 = min((int64_t)a.C.nrows, run * 32 + 32);
    for (int64_t i = run * 32; i < i1; ++i) {
      const int32_t c0 = a.C.rp[i], L = a.C.rp[i + 1] - c0;
      if (L > 255) {
        if (lane == 0) a.rep[i] = -1;
        continue;
      }
      // hash of the relative row
      unsigned long long h = 0x9ae16a3b2f90404full ^ mix64((unsigned long long)(lane + 1) * 0x9e3779b97f4a7c15ull);
      for (int32_t j = lane; j < L; j += 32)
        h = (h ^ (unsigned long long)(uint32_t)(a.C.ci[c0 + j] - (int32_t)i)) * 0x100000001b3ull;
      h = mix64(h + (unsigned long long)lane * 0x632be59bd9b4e019ull + (unsigned long long)L);
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, d);
      if (h == kEmptyKey) h = 0;
      int32_t r = -1;
      for (int q = 0; q < 2 && r < 0; ++q)
        if (memo_h[q] == h && memo[q] >= 0 && same_crow(a.C, (int32_t)i, memo[q])) r = memo[q];
      if (r < 0) {
        uint32_t slot = (uint32_t)(h >> 24) & mask;
        int role = 0;
        if (lane == 0) {
          for (uint32_t probe = 0; probe <= mask && probe < kMaxProbes; ++probe) {
            unsigned long long old = *(volatile unsigned long long*)&a.key[slot];
            if (old == kEmptyKey) old = atomicCAS(&a.key[slot], kEmptyKey, h);
            if (old == kEmptyKey) {
              role = 1;
              break;
            }
            if (old == h) {
              role = 2;
              break;
            }
            slot = (slot + 1) & mask;
          }
        }
        role = __shfl_sync(0xffffffffu, role, 0);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (role == 1) {
          r = (int32_t)i;
          if (lane == 0) {
            a.rep_of_slot[slot] = r;
            __threadfence();
            atomicExch(&a.ready[slot], 1);
          }
        } else if (role == 2) {
          int rdy = 0;
          if (lane == 0) rdy = atomicAdd(&a.ready[slot], 0);
          rdy = __shfl_sync(0xffffffffu, rdy, 0);
          __threadfence();
          const int32_t cand = rdy ? __ldcg(&a.rep_of_slot[slot]) : -1;
          r = (cand >= 0 && same_crow(a.C, (int32_t)i, cand)) ? cand : (int32_t)i;
        } else {
          r = (int32_t)i;  // table full: the row is its own representative
        }
        memo[1] = memo[0];
        memo_h[1] = memo_h[0];
        memo[0] = r;
        memo_h[0] = h;
      }
      if (lane == 0) a.rep[i] = r;
    }
  }
}

// Probes the shape table for the key h: 1 = this row inserted it, 2 = it
// exists, 0 = no room (the row takes the full path).  *slot gets the slot.
__device__ int shape_probe(const ClassArgs& c, unsigned long long h, uint32_t* slot_out) {
  const int lane = threadIdx.x & 31;
  const uint32_t mask = (1u << c.tlog2) - 1u;
  uint32_t slot = (uint32_t)(h >> 24) & mask;
  int role = 0;
  if (lane == 0) {
    for (uint32_t probe = 0; probe <= mask && probe < kMaxProbes; ++probe) {
      unsigned long long old = *(volatile unsigned long long*)&c.skey[slot];
      if (old == kEmptyKey) old = atomicCAS(&c.skey[slot], kEmptyKey, h);
      if (old == kEmptyKey) {
        role = 1;
        break;
      }
      if (old == h) {
        role = 2;
        break;
      }
      slot = (slot + 1) & mask;
    }
  }
  *slot_out = __shfl_sync(0xffffffffu, slot, 0);
  return __shfl_sync(0xffffffffu, role, 0);
}

// One pass over the fine rows.  Most rows of a mesh operator repeat the
// structure of their neighbours, shifted: a row first computes its shape
// (compute_shape: loads only, no sorting or searching) and looks it up in
// the shape table.  The row that inserts a shape computes the program once,
// finds its class in the program table and publishes the shape with that
// class; later rows with an equal shape (compared word by word) take the
// class directly.  Rows whose shape is still being published, or whose
// shape does not fit on chip, compute their program themselves.  Nothing
// waits on another warp; a hash collision can only cost a row the shortcut.
__global__ void __launch_bounds__(kSigWarps * 32) k_class_build(ClassArgs c) {
  __shared__ SigSmem sm;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Each warp takes runs of 32 consecutive fine rows, where neighbouring rows
  // repeat a few shapes, and remembers the last two shapes it resolved (with
  // their classes) in shared memory: most rows match one of them there, with
  // no global atomic and no read of the shared pools.
  int buf = 0;                          // which of the three buffers holds this row's shape
  int memo[2] = {1, 2};                 // buffers of the remembered shapes, most recent first
  unsigned long long memo_h[2] = {kEmptyKey, kEmptyKey};
  int32_t memo_len[2] = {0, 0}, memo_cls[2] = {-2, -2};
  const int64_t warps = (int64_t)gridDim.x * kSigWarps;
  for (int64_t run = (int64_t)blockIdx.x * kSigWarps + w; run * 32 < c.n; run += warps) {
    // one row outside the limits, or a full table, sends the whole plan to the
    // general kernel: nothing left to learn, so every warp stops.  Checked once
    // a run: every warp reading the same word each row would queue on it.
    int stop = 0;
    if (lane == 0) stop = ((volatile int32_t*)c.counters)[2] > 0 || ((volatile int32_t*)c.counters)[3] != 0;
    if (__shfl_sync(0xffffffffu, stop, 0)) return;
    const int64_t I1 = min((int64_t)c.n, run * 32 + 32);
    for (int64_t I = run * 32; I < I1; ++I) {
      if (c.g.P.rp[I + 1] == c.g.P.rp[I]) {  // never visited
        if (lane == 0) c.row_class[I] = -1;
        continue;
      }
      int32_t* sh = sm.shape[w][buf];
      const int slen = compute_shape(c.g, c.crep, (int32_t)I, sh);
      int32_t cls = -2;
      if (slen == -1) {
        cls = -2;  // outside the limits
      } else if (slen < 0) {
        cls = row_program_class(c, (int32_t)I, sm, w);
      } else {
        const unsigned long long h = words_hash(sh, slen);
        int hit = -1;
        for (int q = 0; q < 2 && hit < 0; ++q) {
          if (memo_h[q] != h || memo_len[q] != slen) continue;
          const int32_t* m = sm.shape[w][memo[q]];
          bool same = true;
          for (int x = lane; x < slen; x += 32) same = same && m[x] == sh[x];
          if (__all_sync(0xffffffffu, same)) hit = q;
        }
        if (hit >= 0) {
          cls = memo_cls[hit];
          if (hit == 1) {  // most recent first
            const int tb = memo[0];
            memo[0] = memo[1];
            memo[1] = tb;
            const unsigned long long th = memo_h[0];
            memo_h[0] = memo_h[1];
            memo_h[1] = th;
            const int32_t tl = memo_len[0], tc = memo_cls[0];
            memo_len[0] = memo_len[1];
            memo_cls[0] = memo_cls[1];
            memo_len[1] = tl;
            memo_cls[1] = tc;
          }
        } else {
          uint32_t slot = 0;
          const int role = shape_probe(c, h, &slot);
          if (role == 1) {
            cls = row_program_class(c, (int32_t)I, sm, w);
            int32_t off = -1;
            if (lane == 0) {
              off = (int32_t)atomicAdd(&c.counters[5], slen);
              if ((int64_t)off + slen > c.spool_cap) off = -1;
            }
            off = __shfl_sync(0xffffffffu, off, 0);
            if (off >= 0)
              for (int x = lane; x < slen; x += 32) c.spool[off + x] = sh[x];
            __syncwarp();
            if (lane == 0) {
              c.soff[slot] = off;
              c.scls[slot] = cls;
              __threadfence();  // the shape, its offset and class before the flag
              atomicExch(&c.sready[slot], 1);
            }
          } else if (role == 2) {
            int ready = 0;
            if (lane == 0) ready = atomicAdd(&c.sready[slot], 0);
            ready = __shfl_sync(0xffffffffu, ready, 0);
            __threadfence();
            bool same = false;
            int32_t k = -2;
            if (ready) {
              const int32_t off = __ldcg(&c.soff[slot]);
              k = __ldcg(&c.scls[slot]);
              if (off >= 0 && __ldcg(&c.spool[off]) == sh[0]) {
                same = true;
                for (int x = lane; x < slen; x += 32) same = same && __ldcg(&c.spool[off + x]) == sh[x];
                same = __all_sync(0xffffffffu, same);
              }
            }
            cls = (same && k != -3) ? k : row_program_class(c, (int32_t)I, sm, w);
          } else {
            cls = row_program_class(c, (int32_t)I, sm, w);
          }
          // remember this shape and its class (settled classes only)
          if (cls >= 0 || cls == -2) {
            const int old = memo[1];
            memo[1] = memo[0];
            memo_h[1] = memo_h[0];
            memo_len[1] = memo_len[0];
            memo_cls[1] = memo_cls[0];
            memo[0] = buf;
            memo_h[0] = h;
            memo_len[0] = slen;
            memo_cls[0] = cls;
            buf = old;
          }
        }
      }
      if (lane == 0) {
        c.row_class[I] = cls;
        if (cls == -2) atomicAdd(&c.counters[2], 1);
        if (cls == -3) {
          const int32_t k = atomicAdd(&c.counters[4], 1);
          if (k < c.vcap) c.vlist[k] = (int32_t)I;
        }
      }
      __syncwarp();
    }
  }
}

// nlist >= 0: the rows to settle are vlist[0, nlist); otherwise every row
// marked -3 (the list overflowed).
__global__ void __launch_bounds__(kSigWarps * 32) k_class_verify(ClassArgs c, int32_t nlist) {
  __shared__ SigSmem sm;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t mask = (1u << c.tlog2) - 1u;
  const int64_t total = nlist >= 0 ? nlist : c.n;
  for (int64_t x = (int64_t)blockIdx.x * kSigWarps + w; x < total; x += (int64_t)gridDim.x * kSigWarps) {
    const int64_t I = nlist >= 0 ? c.vlist[x] : x;
    if (c.row_class[I] != -3) continue;
    const int len = compute_sig(c.g, (int32_t)I, sm.sig[w], sm.cand[w], sm.keys[w], c.status);
    int32_t cls = -2;
    if (len > 0) {
      const unsigned long long h = sig_hash(sm.sig[w], len);
      uint32_t slot = (uint32_t)(h >> 20) & mask;
      int32_t found = -1;
      for (uint32_t probe = 0; probe <= mask && probe < kMaxProbes; ++probe) {
        const unsigned long long k = c.tkey[slot];
        if (k == h) {
          found = c.tcls[slot];
          break;
        }
        if (k == kEmptyKey) break;
        slot = (slot + 1) & mask;
      }
      if (found >= 0 && same_program(c, found, sm.sig[w], len)) cls = found;
    }
    if (lane == 0) {
      c.row_class[I] = cls;
      if (cls == -2) atomicAdd(&c.counters[2], 1);
    }
    __syncwarp();
  }
}

// Rows per class (histogram of row_class over the fine rows with a class).
// Lanes holding the same class add once for all of them; with `local` (K
// counters in dynamic shared memory) a CTA counts on chip and then adds its
// totals to cnt.  The loop bound is uniform over the CTA, so every lane
// reaches each match.
__global__ void k_class_rows(const int32_t* __restrict__ row_class, int32_t n, int32_t K, bool local,
                             int32_t* cnt) {
  extern __shared__ int32_t hist[];
  if (local) {
    for (int32_t k = threadIdx.x; k < K; k += blockDim.x) hist[k] = 0;
    __syncthreads();
  }
  int32_t* out = local ? hist : cnt;
  const int lane = threadIdx.x & 31;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = b + threadIdx.x;
    const int32_t k = I < n ? row_class[I] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, k);
    if (k >= 0 && lane == __ffs(peers) - 1) atomicAdd(&out[k], __popc(peers));
  }
  if (local) {
    __syncthreads();
    for (int32_t k = threadIdx.x; k < K; k += blockDim.x)
      if (hist[k]) atomicAdd(&cnt[k], hist[k]);
  }
}

// row_class[I] = perm[row_class[I]] for classed rows.
__global__ void k_class_remap(int32_t* __restrict__ row_class, int32_t n, const int32_t* __restrict__ perm) {
  for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < n; I += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = row_class[I];
    if (k >= 0) row_class[I] = perm[k];
  }
}

// Widest span (last - first fine row) of any chunk's ascending visit list,
// into maxspan[0], and the longest list less one, into maxspan[1].
__global__ void k_chunk_span(const int32_t* __restrict__ fptr, const int32_t* __restrict__ frows,
                             int32_t nch, int32_t* maxspan) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nch;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t f0 = fptr[c], f1 = fptr[c + 1];
    if (f1 > f0) {
      atomicMax(&maxspan[0], frows[f1 - 1] - frows[f0]);
      atomicMax(&maxspan[1], f1 - 1 - f0);
    }
  }
}

// Composite sort key (block of 2^bb consecutive fine rows, class, row): runs
// of one class stay inside a block.  When the rows' span is too wide for the
// key (compact chunks reach many planes of a mesh), the row's rank in the
// ascending list stands for its distance from the first (same order; blocks
// then count visits instead of rows).  Small blocks make the warps working on a
// chunk at the same time read neighbouring rows of A and P (L1 reuse); large
// blocks keep runs long (full warps).  bb is a tuning knob (config).
// The three visit-list kernels below give each chunk a warp, whose lanes
// stride over the chunk's visits.
__global__ void k_visit_keys(const int32_t* __restrict__ fptr, const int32_t* __restrict__ frows,
                             int32_t nch, const int32_t* __restrict__ row_class, int shift,
                             int kBlockBits, bool rank, int32_t* keys) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += nw) {
    const int32_t f0 = fptr[c], f1 = fptr[c + 1];
    if (f0 == f1) continue;
    const int32_t base = frows[f0];  // lists are ascending before this sort
    for (int32_t f = f0 + lane; f < f1; f += 32) {
      const int32_t I = frows[f], d = rank ? f - f0 : I - base;
      keys[f] = ((d >> kBlockBits) << (shift + kBlockBits)) | (row_class[I] << kBlockBits) |
                (d & ((1 << kBlockBits) - 1));
    }
  }
}

// Class-major visit order without a comparison sort: a warp per chunk counts
// its visits per class (a histogram of K counters in shared memory), scans the
// counts, and places the visits batch by batch in their input order -- lanes
// of one class take consecutive slots by rank among their peers -- so each
// class keeps the ascending order the lists come in.  The keys it writes are
// those k_visit_keys forms (class above the position bits), in sorted order:
// the same result as the segmented sort of those keys, when one block covers
// the chunk (visit_block_log2 = 0).
__global__ void k_visit_class_sort(const int32_t* __restrict__ fptr, const int32_t* __restrict__ frows,
                                   int32_t nch, const int32_t* __restrict__ row_class, int32_t K,
                                   int kBlockBits, bool rank, int32_t* __restrict__ keys_out,
                                   int32_t* __restrict__ frows_out) {
  extern __shared__ int32_t hsm[];
  const int lane = threadIdx.x & 31;
  int32_t* hist = hsm + (threadIdx.x >> 5) * K;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int32_t dmask = (1 << kBlockBits) - 1;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += nw) {
    const int32_t f0 = fptr[c], f1 = fptr[c + 1];
    if (f0 == f1) continue;
    for (int32_t k = lane; k < K; k += 32) hist[k] = 0;
    __syncwarp();
    for (int32_t f = f0 + lane; f < f1; f += 32) atomicAdd(&hist[row_class[frows[f]]], 1);
    __syncwarp();
    int32_t carry = f0;  // output positions are absolute
    for (int32_t b = 0; b < K; b += 32) {
      const int32_t v = b + lane < K ? hist[b + lane] : 0;
      int32_t incl = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      if (b + lane < K) hist[b + lane] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    const int32_t basef = frows[f0];
    for (int32_t f = f0; f < f1; f += 32) {
      const bool ok = f + lane < f1;
      const int32_t I = ok ? frows[f + lane] : 0;
      const int32_t cl = ok ? row_class[I] : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, cl);
      const int32_t pos = ok ? hist[cl] + __popc(peers & ((1u << lane) - 1u)) : 0;
      __syncwarp();
      if (ok) {
        const int32_t d = rank ? (f + lane - f0) : (I - basef);
        frows_out[pos] = I;
        keys_out[pos] = (cl << kBlockBits) | (d & dmask);
        if ((peers >> lane) == 1u) hist[cl] += __popc(peers);  // the group's last lane moves the cursor
      }
      __syncwarp();
    }
  }
}

__global__ void k_seg_flags(const int32_t* __restrict__ fptr, int32_t nch, const int32_t* __restrict__ keys,
                            int shift, int kBlockBits, int32_t* flag) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += nw) {
    const int32_t f0 = fptr[c], f1 = fptr[c + 1];
    for (int32_t f = f0 + lane; f < f1; f += 32)
      flag[f] = (f == f0 || (keys[f] >> kBlockBits) != (keys[f - 1] >> kBlockBits)) ? 1 : 0;
  }
}

__global__ void k_seg_fill(const int32_t* __restrict__ fptr, int32_t nch, const int32_t* __restrict__ keys,
                           int shift, int kBlockBits, const int32_t* __restrict__ segid, int32_t* seg_ptr,
                           int32_t* seg_class, int32_t* chunk_seg, int64_t nf) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nch; c += nw) {
    const int32_t f0 = fptr[c], f1 = fptr[c + 1];
    if (lane == 0) chunk_seg[c] = segid[f0];
    for (int32_t f = f0 + lane; f < f1; f += 32)
      if (f == f0 || (keys[f] >> kBlockBits) != (keys[f - 1] >> kBlockBits)) {
        seg_ptr[segid[f]] = f;
        seg_class[segid[f]] = (keys[f] >> kBlockBits) & ((1 << shift) - 1);
      }
  }
}

// Pieces: each run split into groups of at most 32 rows (one per warp step).
__global__ void k_piece_count(const int32_t* __restrict__ seg_ptr, int64_t nseg, int32_t* np) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nseg;
       g += (int64_t)gridDim.x * blockDim.x)
    np[g] = (seg_ptr[g + 1] - seg_ptr[g] + 31) >> 5;
}

__global__ void k_piece_fill(const int32_t* __restrict__ seg_ptr, const int32_t* __restrict__ seg_class,
                             int64_t nseg, const int32_t* __restrict__ poff, int32_t* piece_f0,
                             int32_t* piece_meta) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nseg;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int32_t f0 = seg_ptr[g], len = seg_ptr[g + 1] - f0;
    for (int32_t j = 0; j * 32 < len; ++j) {
      piece_f0[poff[g] + j] = f0 + 32 * j;
      piece_meta[poff[g] + j] = (seg_class[g] << 6) | min(32, len - 32 * j);
    }
  }
}

__global__ void k_chunk_piece(const int32_t* __restrict__ chunk_seg, int32_t nch,
                              const int32_t* __restrict__ poff, int32_t* chunk_piece) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= nch;
       c += (int64_t)gridDim.x * blockDim.x)
    chunk_piece[c] = poff[chunk_seg[c]];
}

}  // namespace

// Builds the classes of the plan's fine rows.  On success with every visited
// row inside the fast-path limits, sets p->fast and fills the pool, the class
// offsets and the max slot count; otherwise leaves p->fast = 0.
int build_classes(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, cudaStream_t s) {
  p->fast = 0;
  if (p->n == 0 || p->nnz_c == 0) return PTAP_OK;
  Scratch sc(&p->mem);
  const int tlog2 = 16;
  const int64_t tcap = (int64_t)1 << tlog2;
  const int64_t pool_cap = (int64_t)1 << 20;
  unsigned long long* tkey = nullptr;
  int32_t *tready = nullptr, *tcls = nullptr, *counters = nullptr, *row_class = nullptr;
  int32_t* class_off = nullptr;
  uint8_t* pool = nullptr;
  PTAP_TRY(sc.get(&tkey, tcap));
  PTAP_TRY(sc.get(&tready, tcap));
  PTAP_TRY(sc.get(&tcls, tcap));
  PTAP_TRY(sc.get(&counters, 8));
  PTAP_TRY(sc.get(&row_class, p->n));
  PTAP_TRY(sc.get(&class_off, tcap + 1));
  PTAP_TRY(sc.get(&pool, pool_cap));
  // representatives of C's rows (k_crow_rep), which the fine rows' shapes name
  int32_t *crep = nullptr, *cready = nullptr, *crslot = nullptr;
  unsigned long long* ckey = nullptr;
  PTAP_TRY(sc.get(&crep, std::max(p->m, 1)));
  PTAP_TRY(sc.get(&ckey, tcap));
  PTAP_TRY(sc.get(&cready, tcap));
  PTAP_TRY(sc.get(&crslot, tcap));
  PTAP_CUDA(cudaMemsetAsync(ckey, 0xff, tcap * sizeof(unsigned long long), s));
  PTAP_CUDA(cudaMemsetAsync(cready, 0, tcap * sizeof(int32_t), s));
  {
    CrowArgs ca{CsrI{p->m, p->m, p->c_rp, p->c_ci}, ckey, cready, crslot, tlog2, crep};
    k_crow_rep<<<num_sms() * 16, 128, 0, s>>>(ca);
    PTAP_LAUNCHED();
  }
  // the shape table in front of the program table (k_class_build)
  const int64_t spool_cap = (int64_t)1 << 22;
  unsigned long long* skey = nullptr;
  int32_t *sready = nullptr, *scls = nullptr, *soff = nullptr, *spool = nullptr;
  PTAP_TRY(sc.get(&skey, tcap));
  PTAP_TRY(sc.get(&sready, tcap));
  PTAP_TRY(sc.get(&scls, tcap));
  PTAP_TRY(sc.get(&soff, tcap));
  PTAP_TRY(sc.get(&spool, spool_cap));
  PTAP_CUDA(cudaMemsetAsync(skey, 0xff, tcap * sizeof(unsigned long long), s));
  PTAP_CUDA(cudaMemsetAsync(sready, 0, tcap * sizeof(int32_t), s));
  PTAP_CUDA(cudaMemsetAsync(tkey, 0xff, tcap * sizeof(unsigned long long), s));
  PTAP_CUDA(cudaMemsetAsync(tready, 0, tcap * sizeof(int32_t), s));
  PTAP_CUDA(cudaMemsetAsync(counters, 0, 8 * sizeof(int32_t), s));
  ClassArgs c;
  c.g = SigGeom{CsrI{A->nrows, A->ncols, A->row_ptr, A->col_idx},
                CsrI{P->nrows, P->ncols, P->row_ptr, P->col_idx}, CsrI{p->m, p->m, p->c_rp, p->c_ci}};
  c.n = p->n;
  c.tkey = tkey;
  c.tready = tready;
  c.tcls = tcls;
  c.tlog2 = tlog2;
  c.pool = pool;
  c.pool_cap = pool_cap;
  c.class_off = class_off;
  c.counters = counters;
  c.row_class = row_class;
  c.status = p->status;
  c.skey = skey;
  c.sready = sready;
  c.scls = scls;
  c.spool = spool;
  c.soff = soff;
  c.spool_cap = spool_cap;
  c.crep = crep;
  c.vcap = 1 << 20;
  PTAP_TRY(sc.get(&c.vlist, c.vcap));
  // latency-bound warp-per-row work: fill the SMs (16 CTAs of 4 warps each)
  const int grid = num_sms() * 16;
  PhaseRange r_build("ptap: class signatures", s);
  k_class_build<<<grid, kSigWarps * 32, 0, s>>>(c);
  PTAP_LAUNCHED();
  int32_t h[5];
  PTAP_CUDA(cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  if (h[2] > 0 || h[3]) return PTAP_OK;  // some row outside the limits, or table full
  if (h[4] > 0) {  // rows that met their key before its program was published
    const int32_t nlist = h[4] <= c.vcap ? h[4] : -1;
    k_class_verify<<<nlist >= 0 ? (int)std::max<int64_t>(1, std::min<int64_t>(grid, ceil_div(nlist, kSigWarps))) : grid,
                     kSigWarps * 32, 0, s>>>(c, nlist);
    PTAP_LAUNCHED();
    PTAP_CUDA(cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, s));
    PTAP_CUDA(cudaStreamSynchronize(s));
    if (h[2] > 0 || h[3]) return PTAP_OK;
  }
  const int32_t K = h[0];
  const int32_t pool_used = h[1];
  // Canonical class numbering.  Ids from the concurrent publication above
  // differ between runs, and the visit order inside a chunk is class-major by
  // id; renumbering by (rows ascending, program bytes) makes plans for the
  // same patterns identical and their numeric times reproducible.  Of the
  // orders measured (rows ascending or descending, program bytes, estimated
  // cost per row either way), rows ascending -- the few boundary classes
  // first, the populous interior classes last -- ran fastest, by 6-10%.
  {
    std::vector<int32_t> hoff(K), hrows(K);
    std::vector<uint8_t> hpool(std::max(pool_used, 1));
    int32_t* cnt = nullptr;
    PTAP_TRY(sc.get(&cnt, std::max(K, 1)));
    PTAP_CUDA(cudaMemsetAsync(cnt, 0, std::max(K, 1) * sizeof(int32_t), s));
    const bool local = K <= 12288;  // counters within the default 48 KB of shared memory
    k_class_rows<<<local ? num_sms() * 4 : grid, 256, local ? (size_t)K * sizeof(int32_t) : 0, s>>>(
        row_class, p->n, K, local, cnt);
    PTAP_LAUNCHED();
    PTAP_CUDA(cudaMemcpyAsync(hoff.data(), class_off, K * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PTAP_CUDA(cudaMemcpyAsync(hrows.data(), cnt, K * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PTAP_CUDA(cudaMemcpyAsync(hpool.data(), pool, pool_used, cudaMemcpyDeviceToHost, s));
    PTAP_CUDA(cudaStreamSynchronize(s));
    auto prog = [&](int k) { return hpool.data() + hoff[k]; };
    auto len = [&](int k) { return program_length(prog(k)); };
    std::vector<int32_t> order(K), perm(K), noff(K);
    for (int k = 0; k < K; ++k) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
      if (hrows[x] != hrows[y]) return hrows[x] < hrows[y];
      return std::lexicographical_compare(prog(x), prog(x) + len(x), prog(y), prog(y) + len(y));
    });
    for (int k = 0; k < K; ++k) {
      perm[order[k]] = k;
      noff[k] = hoff[order[k]];
    }
    int32_t* dperm = nullptr;
    PTAP_TRY(sc.get(&dperm, std::max(K, 1)));
    PTAP_CUDA(cudaMemcpyAsync(dperm, perm.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PTAP_CUDA(cudaMemcpyAsync(class_off, noff.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_class_remap<<<grid, 256, 0, s>>>(row_class, p->n, dperm);
    PTAP_LAUNCHED();
    PTAP_CUDA(cudaStreamSynchronize(s));
  }
  // composite visit keys need class (bits) + span of each chunk's fine rows
  int kb = 1;
  while ((1 << kb) <= K) ++kb;
  const int shift = kb;  // class field width
  PTAP_CUDA(cudaMemsetAsync(counters, 0, 2 * sizeof(int32_t), s));
  k_chunk_span<<<grid, 256, 0, s>>>(p->chunk_fptr, p->chunk_frows, p->nchunks, counters);
  PTAP_LAUNCHED();
  int32_t spans[2] = {0, 0};
  PTAP_CUDA(cudaMemcpyAsync(spans, counters, sizeof(spans), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  int32_t maxspan = spans[0];
  bool rank = false;
  {
    int need = 0;
    while (((int64_t)1 << need) <= (int64_t)maxspan) ++need;
    if (need + kb > 31) {
      maxspan = spans[1];
      rank = true;
    }
  }
  // key bits: block (d >> bb) | class (kb bits) | d & (2^bb - 1), all below bit 31;
  // bb defaults to the whole chunk span (class-major order)
  int kBlockBits = p->cfg.visit_block_log2 > 0 ? p->cfg.visit_block_log2 : 31 - kb;
  {
    int need = 0;
    while (((int64_t)1 << need) <= (int64_t)maxspan) ++need;
    if (p->cfg.visit_block_log2 <= 0) kBlockBits = std::min(kBlockBits, std::max(need, 1));
  }
  if (kBlockBits > 31 - kb) kBlockBits = 31 - kb;
  if (shift < 1 || kBlockBits < 1 ||
      ((int64_t)maxspan >> kBlockBits) >= ((int64_t)1 << (31 - kb - kBlockBits)))
    return PTAP_OK;
  int32_t *keys = nullptr, *flag = nullptr, *segid = nullptr;
  PTAP_TRY(sc.get(&keys, p->nfrows));
  PTAP_TRY(sc.get(&flag, p->nfrows));
  PTAP_TRY(sc.get(&segid, p->nfrows + 1));
  {
    PhaseRange r_sort("ptap: visit order sort", s);
    constexpr int32_t kCountSortMaxClasses = 2048;
    if (p->cfg.visit_block_log2 <= 0 && K <= kCountSortMaxClasses) {
      // class-major order by counting (k_visit_class_sort) into a new visit list
      int32_t* sorted = nullptr;
      PTAP_TRY(p->mem.get_n(&sorted, std::max<int64_t>(p->nfrows, 1)));
      const int warps = 4;
      const size_t smem = (size_t)warps * K * sizeof(int32_t);
      PTAP_TRY(grow_smem_limit((const void*)k_visit_class_sort, (int)smem));
      k_visit_class_sort<<<grid, warps * 32, smem, s>>>(p->chunk_fptr, p->chunk_frows, p->nchunks, row_class, K,
                                                        kBlockBits, rank, keys, sorted);
      PTAP_LAUNCHED();
      p->mem.put(p->chunk_frows);
      p->chunk_frows = sorted;
    } else {
      k_visit_keys<<<grid, 256, 0, s>>>(p->chunk_fptr, p->chunk_frows, p->nchunks, row_class, shift,
                                        kBlockBits, rank, keys);
      PTAP_LAUNCHED();
      PTAP_TRY(segmented_sort(p->mem, p->chunk_fptr, p->nchunks, keys, p->chunk_frows, -1, s));
    }
  }
  k_seg_flags<<<grid, 256, 0, s>>>(p->chunk_fptr, p->nchunks, keys, shift, kBlockBits, flag);
  PTAP_LAUNCHED();
  int64_t nseg = 0;
  PTAP_TRY(exclusive_scan(p->mem, flag, segid, p->nfrows, &nseg, s));
  int32_t *seg_ptr = nullptr, *seg_class = nullptr, *chunk_seg = nullptr, *np = nullptr, *poff = nullptr;
  PTAP_TRY(sc.get(&seg_ptr, nseg + 1));
  PTAP_TRY(sc.get(&seg_class, std::max<int64_t>(nseg, 1)));
  PTAP_TRY(sc.get(&chunk_seg, (int64_t)p->nchunks + 1));
  k_seg_fill<<<grid, 256, 0, s>>>(p->chunk_fptr, p->nchunks, keys, shift, kBlockBits, segid, seg_ptr,
                                  seg_class, chunk_seg, p->nfrows);
  PTAP_LAUNCHED();
  const int32_t endv[2] = {(int32_t)p->nfrows, (int32_t)nseg};
  PTAP_CUDA(cudaMemcpyAsync(seg_ptr + nseg, &endv[0], sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaMemcpyAsync(chunk_seg + p->nchunks, &endv[1], sizeof(int32_t), cudaMemcpyHostToDevice, s));
  // pieces of at most 32 rows, and each chunk's first piece
  PTAP_TRY(sc.get(&np, nseg + 1));
  PTAP_TRY(sc.get(&poff, nseg + 1));
  k_piece_count<<<grid, 256, 0, s>>>(seg_ptr, nseg, np);
  PTAP_LAUNCHED();
  int64_t npieces = 0;
  PTAP_TRY(exclusive_scan(p->mem, np, poff, nseg, &npieces, s));
  PTAP_TRY(p->mem.get_n(&p->piece_f0, std::max<int64_t>(npieces, 1)));
  PTAP_TRY(p->mem.get_n(&p->piece_meta, std::max<int64_t>(npieces, 1)));
  PTAP_TRY(p->mem.get_n(&p->chunk_piece, (int64_t)p->nchunks + 1));
  k_piece_fill<<<grid, 256, 0, s>>>(seg_ptr, seg_class, nseg, poff, p->piece_f0, p->piece_meta);
  PTAP_LAUNCHED();
  k_chunk_piece<<<grid, 256, 0, s>>>(chunk_seg, p->nchunks, poff, p->chunk_piece);
  PTAP_LAUNCHED();
  p->npieces = npieces;
  // pool and offsets (offsets compacted by class id)
  PTAP_TRY(p->mem.get_n(&p->class_pool, (int64_t)pool_used + kFastSigCap + 32));
  PTAP_TRY(p->mem.get_n(&p->class_off, (int64_t)K + 1));
  PTAP_CUDA(cudaMemcpyAsync(p->class_pool, pool, pool_used, cudaMemcpyDeviceToDevice, s));
  PTAP_CUDA(cudaMemcpyAsync(p->class_off, class_off, K * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  // max r over classes decides the kernel variant
  std::vector<uint8_t> hp(pool_used);
  std::vector<int32_t> ho(K);
  PTAP_CUDA(cudaMemcpyAsync(hp.data(), pool, pool_used, cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaMemcpyAsync(ho.data(), class_off, K * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  int maxr = 0, maxlen = 0, maxa = 0;
  for (int32_t k = 0; k < K; ++k) {
    const uint8_t* g = hp.data() + ho[k];
    maxr = std::max<int>(maxr, g[1]);
    maxa = std::max<int>(maxa, g[0]);
    maxlen = std::max(maxlen, program_length(g));
  }
  p->nclasses = K;
  p->nseg = (int32_t)nseg;
  p->class_maxr = maxr;
  p->class_maxa = maxa;
  p->class_maxlen = maxlen;
  p->fast = 1;
  return PTAP_OK;
}

}  // namespace ptap
