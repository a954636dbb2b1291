// Batched in-place complex FFTs on lines held in shared memory (sm_103a).
//
// The Fourier transforms F, F^-1 of Section 2 (Algorithm 1) are the bulk of
// every fixed-point step.  A line of length N = N1 * N2 is transformed in two
// register steps with one shared-memory exchange between them:
//
//   forward  x[n1*N2 + n2]  ->  X[k1 + N1*k2]  stored at slot k1*N2 + k2
//     step 1: for each n2, a length-N1 DFT over n1 (stride N2), times the
//             twiddle W_N^(n2*k1), written back to the slots it was read from;
//     step 2: for each k1, a length-N2 DFT over the contiguous block k1*N2+.
//   inverse  takes that digit-transposed slot order back to natural order by
//            running the two steps in the opposite order with conjugates.
//
// Keeping spectra in slot order means no permutation pass is ever needed:
// the Green-operator step maps a slot to its frequency arithmetically.
//
// Register DFTs of length 1, 2, 3, 4, 6, 8, 12, 16 are written out with exact
// constants; twiddles W_N^m come from host tables computed in double.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpm {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// multiply by -i (forward kernel sign) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

constexpr float kSqrtHalf = 0.707106781186547524400844362105f;
constexpr float kCosPi8 = 0.923879532511286756128183189397f;
constexpr float kSinPi8 = 0.382683432365089771728459984030f;

// exp(-+ 2 pi i m / 16) for the in-register 16-point transform
template <bool INV>
__device__ __forceinline__ float2 w16(int m) {
  float c, s;
  switch (m & 15) {
    case 0: c = 1.f; s = 0.f; break;
    case 1: c = kCosPi8; s = kSinPi8; break;
    case 2: c = kSqrtHalf; s = kSqrtHalf; break;
    case 3: c = kSinPi8; s = kCosPi8; break;
    case 4: c = 0.f; s = 1.f; break;
    case 6: c = -kSqrtHalf; s = kSqrtHalf; break;
    case 9: c = -kCosPi8; s = -kSinPi8; break;
    default: c = 0.f; s = 0.f; break;   // not used by the 4x4 split
  }
  return INV ? make_float2(c, s) : make_float2(c, -s);
}

template <int R, bool INV>
struct RegDft;

template <bool INV>
struct RegDft<1, INV> {
  __device__ __forceinline__ static void run(float2*) {}
};

template <bool INV>
struct RegDft<2, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct RegDft<4, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <bool INV>
struct RegDft<8, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    RegDft<4, INV>::run(e);
    RegDft<4, INV>::run(o);
    // o1 *= W8^1, o2 *= W8^2, o3 *= W8^3
    {
      float2 a = o[1];
      o[1] = INV ? make_float2(kSqrtHalf * (a.x - a.y), kSqrtHalf * (a.x + a.y))
                 : make_float2(kSqrtHalf * (a.x + a.y), kSqrtHalf * (a.y - a.x));
      o[2] = mul_mi<INV>(o[2]);
      a = o[3];
      o[3] = INV ? make_float2(kSqrtHalf * (-a.x - a.y), kSqrtHalf * (a.x - a.y))
                 : make_float2(kSqrtHalf * (-a.x + a.y), kSqrtHalf * (-a.x - a.y));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
};

constexpr float kSqrt3Half = 0.866025403784438646763723170753f;

// exp(-+ 2 pi i m / 12): multiples of 30 degrees, exact constants
template <bool INV>
__device__ __forceinline__ float2 w12(int m) {
  float c, s;
  switch (m % 12) {
    case 0: c = 1.f; s = 0.f; break;
    case 1: c = kSqrt3Half; s = 0.5f; break;
    case 2: c = 0.5f; s = kSqrt3Half; break;
    case 3: c = 0.f; s = 1.f; break;
    case 4: c = -0.5f; s = kSqrt3Half; break;
    case 5: c = -kSqrt3Half; s = 0.5f; break;
    case 6: c = -1.f; s = 0.f; break;
    case 7: c = -kSqrt3Half; s = -0.5f; break;
    case 8: c = -0.5f; s = -kSqrt3Half; break;
    case 9: c = 0.f; s = -1.f; break;
    case 10: c = 0.5f; s = -kSqrt3Half; break;
    default: c = kSqrt3Half; s = -0.5f; break;
  }
  return INV ? make_float2(c, s) : make_float2(c, -s);
}

template <bool INV>
struct RegDft<3, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 a = v[0], b = v[1], c = v[2];
    const float2 t = cadd(b, c);
    const float2 m = make_float2(a.x - 0.5f * t.x, a.y - 0.5f * t.y);
    const float2 d = make_float2(kSqrt3Half * (b.x - c.x), kSqrt3Half * (b.y - c.y));
    v[0] = cadd(a, t);
    // forward: X1 = m - i d, X2 = m + i d (inverse: the conjugate pattern)
    v[1] = INV ? make_float2(m.x - d.y, m.y + d.x) : make_float2(m.x + d.y, m.y - d.x);
    v[2] = INV ? make_float2(m.x + d.y, m.y - d.x) : make_float2(m.x - d.y, m.y + d.x);
  }
};

// Two-level in-register DFT of length A * B: A-point DFTs over the stride-B
// subsequences, twiddles W_(A B)^(n2 k1), B-point DFTs; natural output order.
// TW(m) returns W_(A B)^m for the table used by the length.
template <int A, int B, bool INV, int TWN>
__device__ __forceinline__ void reg_dft_2level(float2* v) {
  float2 y[B][A];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) {
    float2 t[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) t[n1] = v[n1 * B + n2];
    RegDft<A, INV>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      if (n2 && k1) {
        const float2 w = TWN == 16 ? w16<INV>(n2 * k1) : w12<INV>((12 / (A * B)) * n2 * k1);
        y[n2][k1] = cmul(t[k1], w);
      } else {
        y[n2][k1] = t[k1];
      }
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    float2 t[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2][k1];
    RegDft<B, INV>::run(t);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = t[k2];
  }
}

template <bool INV>
struct RegDft<16, INV> {
  __device__ __forceinline__ static void run(float2* v) { reg_dft_2level<4, 4, INV, 16>(v); }
};
template <bool INV>
struct RegDft<6, INV> {
  __device__ __forceinline__ static void run(float2* v) { reg_dft_2level<3, 2, INV, 12>(v); }
};
template <bool INV>
struct RegDft<12, INV> {
  __device__ __forceinline__ static void run(float2* v) { reg_dft_2level<4, 3, INV, 12>(v); }
};

// Split of a line length N = N1 * N2 into the two register steps.  One
// definition serves device templates and host-side table builders.
// Register DFT lengths: 1, 2, 3, 4, 6, 8, 12, 16.  Lines up to 256 = 2^a 3^b.
__host__ __device__ constexpr int split_n1(int N) {
  return N <= 16 ? N : (N == 24 || N == 32 || N == 64 ? 8 : 16);
}
__host__ __device__ constexpr int split_n2(int N) { return N / split_n1(N); }
__host__ __device__ constexpr bool fft_size_ok(int N) {
  return N == 1 || N == 2 || N == 3 || N == 4 || N == 6 || N == 8 || N == 12 || N == 16 ||
         N == 24 || N == 32 || N == 48 || N == 64 || N == 96 || N == 128 || N == 256;
}

template <int N>
struct Split {
  static constexpr int N1 = split_n1(N), N2 = split_n2(N);
};

// Slot of frequency k in the digit-transposed order, and its inverse.
template <int N>
__host__ __device__ __forceinline__ int slot_of(int k) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  return (k % N1) * N2 + k / N1;
}
template <int N>
__host__ __device__ __forceinline__ int freq_of(int s) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  return s / N2 + N1 * (s % N2);
}
__host__ __device__ inline int freq_of_rt(int N, int s) {
  const int N2 = split_n2(N);
  return s / N2 + split_n1(N) * (s % N2);
}

// In-place FFT of `nlines` lines of length N in shared memory; element i of
// line b sits at buf[b * lstride + i * estride].  `tw` holds W_N^(n2*k1) at
// index n2*N1 + k1 (forward sign).  Forward: natural -> slot order; inverse:
// slot order -> natural.  Unnormalised.  Every thread of the block must call
// it; it ends with __syncthreads().
template <int N, bool INV, int NLINES, int LSTRIDE, int ESTRIDE>
__device__ __forceinline__ void smem_fft(float2* buf, const float2* tw) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  // compile-time shape: task splits are mul-shifts, element offsets immediates
  constexpr int nlines = NLINES, lstride = LSTRIDE, estride = ESTRIDE;
  if (N == 1) return;
  if (!INV) {
    for (int t = threadIdx.x; t < nlines * N2; t += blockDim.x) {
      const int b = t % nlines, n2 = t / nlines;
      float2* p = buf + b * lstride + n2 * estride;
      float2 v[N1];
#pragma unroll
      for (int i = 0; i < N1; ++i) v[i] = p[i * N2 * estride];
      RegDft<N1, false>::run(v);
      if (N2 > 1) {
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], tw[n2 * N1 + k1]);
      }
#pragma unroll
      for (int i = 0; i < N1; ++i) p[i * N2 * estride] = v[i];
    }
    __syncthreads();
    if (N2 > 1) {
      for (int t = threadIdx.x; t < nlines * N1; t += blockDim.x) {
        const int b = t % nlines, k1 = t / nlines;
        float2* p = buf + b * lstride + k1 * N2 * estride;
        float2 v[N2];
#pragma unroll
        for (int i = 0; i < N2; ++i) v[i] = p[i * estride];
        RegDft<N2, false>::run(v);
#pragma unroll
        for (int i = 0; i < N2; ++i) p[i * estride] = v[i];
      }
      __syncthreads();
    }
  } else {
    if (N2 > 1) {
      for (int t = threadIdx.x; t < nlines * N1; t += blockDim.x) {
        const int b = t % nlines, k1 = t / nlines;
        float2* p = buf + b * lstride + k1 * N2 * estride;
        float2 v[N2];
#pragma unroll
        for (int i = 0; i < N2; ++i) v[i] = p[i * estride];
        RegDft<N2, true>::run(v);
#pragma unroll
        for (int n2 = 1; n2 < N2; ++n2) v[n2] = cmulc(v[n2], tw[n2 * N1 + k1]);
#pragma unroll
        for (int i = 0; i < N2; ++i) p[i * estride] = v[i];
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < nlines * N2; t += blockDim.x) {
      const int b = t % nlines, n2 = t / nlines;
      float2* p = buf + b * lstride + n2 * estride;
      float2 v[N1];
#pragma unroll
      for (int i = 0; i < N1; ++i) v[i] = p[i * N2 * estride];
      RegDft<N1, true>::run(v);
#pragma unroll
      for (int i = 0; i < N1; ++i) p[i * N2 * estride] = v[i];
    }
    __syncthreads();
  }
}

}  // namespace rpm
