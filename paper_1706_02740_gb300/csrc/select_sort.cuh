// Sorting and medians for the selections, on integer keys.
//
// Records are ordered by larger magnitude first, then the smaller frequency (then the index, so
// that the order is total).  Magnitudes are compared through the bit patterns of non-negative IEEE
// doubles, which are monotone in their values: FP64 comparisons would run on the FP64 pipe, which
// GB300 provisions at a small fraction of its integer and FP32 rates.
//
// reg_bitonic sorts 1024 E records held E per thread (element e = u * 1024 + threadIdx.x): the
// compare-exchange stages whose partner distance j is >= 1024 stay inside a thread, j < 32 use
// warp shuffles, and only 32 <= j < 1024 go through shared memory.
#pragma once

#include <stdint.h>

namespace sft {

constexpr int kSortThreads = 1024;
constexpr int kSortCap = 8192;       // records one CTA sorts (E = 8)
constexpr int kRankThreads = 256;

struct Rec {
  uint64_t m;   // magnitude key
  int64_t w;    // frequency
  int32_t ix;   // payload index
  int32_t pad;
};
constexpr int kSortSmem = kSortCap * (int)sizeof(Rec);

// magnitude key of a non-negative double
__device__ __forceinline__ uint64_t mag_key(double m2) {
  return (uint64_t)__double_as_longlong(m2);
}

// a precedes b: larger magnitude first, then the smaller frequency
__device__ __forceinline__ bool precedes(uint64_t ma, int64_t wa, uint64_t mb, int64_t wb) {
  return ma > mb || (ma == mb && wa < wb);
}

__device__ __forceinline__ bool rec_first(const Rec& a, const Rec& b) {
  return a.m > b.m || (a.m == b.m && (a.w < b.w || (a.w == b.w && a.ix < b.ix)));
}

__device__ __forceinline__ Rec pad_rec(int e) {
  Rec r;
  r.m = 0;
  r.w = INT64_MAX;
  r.ix = INT32_MAX - e;
  r.pad = 0;
  return r;
}

__device__ __forceinline__ Rec shfl_xor_rec(const Rec& r, int j) {
  Rec o;
  o.m = __shfl_xor_sync(0xffffffffu, (unsigned long long)r.m, j);
  o.w = __shfl_xor_sync(0xffffffffu, (long long)r.w, j);
  o.ix = __shfl_xor_sync(0xffffffffu, r.ix, j);
  o.pad = 0;
  return o;
}

// What element e keeps after comparing with its partner e ^ j inside a merge block of size k.
__device__ __forceinline__ Rec keep_of(const Rec& mine, const Rec& other, int e, int j, int k) {
  const int p = e ^ j;
  const bool ascending = ((e < p ? e : p) & k) == 0;
  const bool want_first = (e < p) == ascending;
  return (want_first == rec_first(mine, other)) ? mine : other;
}

template <int E>
__device__ __forceinline__ void reg_bitonic(Rec (&r)[E], Rec* smem) {
  constexpr int NT = 1024 * E;
  const int t = threadIdx.x;
  for (int k = 2; k <= NT; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 1024) {
        const int ju = j >> 10;
#pragma unroll
        for (int u = 0; u < E; ++u) {
#pragma unroll
          for (int v = u + 1; v < E; ++v) {
            if ((u ^ v) == ju) {
              const int e = u * 1024 + t;          // e < its partner
              const bool ascending = (e & k) == 0;
              if (ascending != rec_first(r[u], r[v])) {
                const Rec tmp = r[u];
                r[u] = r[v];
                r[v] = tmp;
              }
            }
          }
        }
      } else if (j >= 32) {
#pragma unroll
        for (int u = 0; u < E; ++u) smem[u * 1024 + t] = r[u];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < E; ++u) {
          const int e = u * 1024 + t;
          r[u] = keep_of(r[u], smem[e ^ j], e, j, k);
        }
        __syncthreads();
      } else {
#pragma unroll
        for (int u = 0; u < E; ++u) r[u] = keep_of(r[u], shfl_xor_rec(r[u], j), u * 1024 + t, j, k);
      }
    }
  }
}

// Sorts smem[0 .. 1024 E) in place (callers fill unused slots with pad_rec); all kSortThreads
// threads of the CTA must call it.
template <int E>
__device__ __forceinline__ void sort_smem_E(Rec* smem) {
  Rec r[E];
#pragma unroll
  for (int u = 0; u < E; ++u) r[u] = smem[u * 1024 + threadIdx.x];
  __syncthreads();
  reg_bitonic<E>(r, smem);
#pragma unroll
  for (int u = 0; u < E; ++u) smem[u * 1024 + threadIdx.x] = r[u];
  __syncthreads();
}

// Number of slots (1024 E) the sort of n records uses.
__device__ __forceinline__ int sort_slots(int n) {
  return n <= 1024 ? 1024 : (n <= 2048 ? 2048 : (n <= 4096 ? 4096 : 8192));
}

__device__ __forceinline__ void sort_smem(Rec* smem, int n) {
  const int slots = sort_slots(n);
  if (slots == 1024) sort_smem_E<1>(smem);
  else if (slots == 2048) sort_smem_E<2>(smem);
  else if (slots == 4096) sort_smem_E<4>(smem);
  else sort_smem_E<8>(smem);
}

// Order-preserving maps of floating-point values to unsigned integers (for medians without
// floating-point comparisons).
__device__ __forceinline__ uint64_t order_key(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ uint32_t order_key(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b >> 31) ? ~b : (b | 0x80000000u);
}

// Median of n <= CAP values (the middle one for odd n, the mean of the two middle ones, in FP64,
// for even n), sorting by integer keys.
template <int CAP, typename T>
__device__ __forceinline__ double median_of(const T* a, int n) {
  decltype(order_key(a[0])) k[CAP];
  int ix[CAP];
  for (int i = 0; i < n; ++i) { k[i] = order_key(a[i]); ix[i] = i; }
  for (int i = 1; i < n; ++i) {
    const auto v = k[i];
    const int xv = ix[i];
    int j = i - 1;
    while (j >= 0 && k[j] > v) { k[j + 1] = k[j]; ix[j + 1] = ix[j]; --j; }
    k[j + 1] = v;
    ix[j + 1] = xv;
  }
  return (n & 1) ? (double)a[ix[n / 2]] : 0.5 * ((double)a[ix[n / 2 - 1]] + (double)a[ix[n / 2]]);
}

}  // namespace sft
