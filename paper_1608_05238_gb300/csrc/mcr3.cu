// mcr3.cu -- the 3D form of the harmonic radiance Monte Carlo (include/mcr3.h): voxel transport
// with the 3D Henyey-Greenstein phase function, spherical-harmonic track-length tallies in 64-bit
// fixed point, the adjoint run turned by pi, and the voxelwise H, eps and functional gradients.
//
// Kernel layout follows the 2D transport: persistent warps, one packet per lane, a global packet
// counter; each lane keeps the real spherical harmonics Y_lm of its current flight direction in
// a shared-memory row, and every voxel segment is deposited by the whole warp, 32 coefficients
// per reduction instruction, into rows of tally_row_words((L+1)^2) words per voxel.
#include <math.h>
#include <math_constants.h>

#include <mutex>

#include "../../include/mcr3.h"
#include "mcr_internal.h"
#include "mcr_rng.cuh"

namespace mcr {
namespace {

constexpr unsigned kFull3 = 0xFFFFFFFFu;
constexpr int kMaxC3 = (MCR3_MAX_L + 1) * (MCR3_MAX_L + 1);
constexpr int kThreads3 = 128;

struct Transport3Params {
  int nx, ny, nz;
  float dx, g;
  int L, C, Cpad, row_stride;
  const float4 *mu;  // packed (mu_a, mu_s, 1/mu_a, 1/mu_s) per voxel
  unsigned long long *tally;
  const unsigned long long *cdf;  // volumetric source: inclusive prefix of quantised |q|
  const float *q;
  int kind;  // MCR_PENCIL, MCR_ISO_POINT, or -1: volumetric
  float x0, y0, z0, ux0, uy0, uz0;
  unsigned key0, key1;
  unsigned long long first_packet, n_packets;
  unsigned max_scatter, max_events;
  float w_threshold, rr_p, rr_inv_p, qscale;
  float nlm[kMaxC3];  // N_lm (times sqrt 2 for m != 0) at index l^2 + l + |m|
  float rinv[MCR3_MAX_L + 1];  // 1 / k
  unsigned long long *work;
  DevStats *stats;
  unsigned *flags;
};

// Real orthonormal spherical harmonics of the unit direction u into row[c], c = l^2 + l + m:
// Y_lm = N_lm Q_l^|m|(u_z) Re/Im[(u_x + i u_y)^|m|], with P_l^m = (1 - u_z^2)^{m/2} Q_l^m and
// Q_m^m = (2m-1)!!, Q_{m+1}^m = (2m+1) u_z Q_m^m, (l - m) Q_l^m = (2l-1) u_z Q_{l-1}^m - (l+m-1) Q_{l-2}^m.
__device__ __forceinline__ void sh_row(const Transport3Params &p, float ux, float uy, float uz, float *row) {
  float cr = 1.f, ci = 0.f;  // (u_x + i u_y)^m
  float qmm = 1.f;           // Q_m^m
  for (int m = 0; m <= p.L; ++m) {
    float q2 = 0.f, q1 = qmm;
    for (int l = m; l <= p.L; ++l) {
      float ql;
      if (l == m)
        ql = qmm;
      else if (l == m + 1)
        ql = (2.f * m + 1.f) * uz * qmm;
      else
        ql = ((2.f * l - 1.f) * uz * q1 - (l + m - 1.f) * q2) * p.rinv[l - m];
      if (l > m) {
        q2 = q1;
        q1 = ql;
      }
      const int c0 = l * l + l;
      const float a = p.nlm[c0 + m] * ql;
      if (m == 0) {
        row[c0] = a;
      } else {
        row[c0 + m] = a * cr;
        row[c0 - m] = a * ci;
      }
    }
    const float nr = cr * ux - ci * uy, ni = cr * uy + ci * ux;
    cr = nr;
    ci = ni;
    qmm *= 2.f * m + 1.f;
  }
}

// cos of a 3D Henyey-Greenstein scattering angle by the inverse CDF at u
__device__ __forceinline__ float hg3_cos(float g, float u) {
  if (fabsf(g) < 1e-6f) return 2.f * u - 1.f;
  const float f = (1.f - g * g) / (1.f - g + 2.f * g * u);
  return fminf(fmaxf((1.f + g * g - f * f) / (2.f * g), -1.f), 1.f);
}

// Turn u by polar cos ct and azimuth 2 pi v about itself, in the orthonormal frame of Duff et al.
// (JCGT 2017), then renormalise.
__device__ __forceinline__ void turn(float &ux, float &uy, float &uz, float ct, float v) {
  const float sgn = uz >= 0.f ? 1.f : -1.f;
  const float a = -1.f / (sgn + uz), b = ux * uy * a;
  const float t1x = 1.f + sgn * ux * ux * a, t1y = sgn * b, t1z = -sgn * ux;
  const float t2x = b, t2y = sgn + uy * uy * a, t2z = -uy;
  const float st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
  float sp, cp;
  sincospif(2.f * v, &sp, &cp);
  float nx = ct * ux + st * (cp * t1x + sp * t2x);
  float ny = ct * uy + st * (cp * t1y + sp * t2y);
  float nz = ct * uz + st * (cp * t1z + sp * t2z);
  const float inv = rsqrtf(nx * nx + ny * ny + nz * nz);
  ux = nx * inv;
  uy = ny * inv;
  uz = nz * inv;
}

__device__ __forceinline__ int pick_voxel(const unsigned long long *__restrict__ cdf, int n, unsigned long long total,
                                          unsigned w0, unsigned w1) {
  const unsigned long long r48 = ((unsigned long long)w0 << 16) | (unsigned long long)(w1 >> 16);
  const unsigned long long target = __umul64hi(r48 << 16, total);
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = lo + ((hi - lo) >> 1);
    if (__ldg(cdf + mid) > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ float clamp3(float v, float dx) { return fminf(fmaxf(v, 0.f), dx); }

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull3, v, o);
  return v;
}

// NCH: 32-lane passes per voxel row ((L+1)^2 <= 32 NCH).  MERGE: a collision segment of a packet
// that survives the collision is deposited together with the next flight's first segment (the
// same voxel), the two rows' products rounded separately and added as integers -- the tally is
// bit-identical, with one warp pass instead of two; each lane then keeps two rows (the previous
// flight's and the current one) in shared memory.
template <int NCH, bool MERGE>
__global__ void __launch_bounds__(kThreads3, 8) k_transport3(const __grid_constant__ Transport3Params p) {
  extern __shared__ float rows3[];
  constexpr int kRows = MERGE ? 2 : 1;
  const int lane = threadIdx.x & 31;
  float *const myrows = rows3 + (size_t)threadIdx.x * kRows * p.row_stride;
  const float *const warprows = rows3 + (size_t)(threadIdx.x & ~31) * kRows * p.row_stride;
  int rb = 0;         // MERGE: which of the lane's two rows holds the current flight's harmonics
  float carry = 0.f;  // MERGE: deferred collision segment (track weight x 2^q), previous row
  if (*p.flags & kFlagMedium) return;
  const int nvox = p.nx * p.ny * p.nz;
  const float dx = p.dx;

  bool alive = false, exhausted = false;
  unsigned long long pid = 0;
  float fx = 0.f, fy = 0.f, fz = 0.f, ux = 0.f, uy = 0.f, uz = 1.f, W = 0.f, W0 = 1.f, tau = 0.f;
  float inv_ax = 0.f, inv_ay = 0.f, inv_az = 0.f;  // 1 / |u| per axis, set per flight
  int ix = 0, iy = 0, iz = 0;
  unsigned flight = 0, nscat = 0, cu1 = 0, cu2 = 0, cu3 = 0;
  // lane counters in 32 bits (segments bound all of them but the launches, which are < 2^26 per
  // call); the warp flushes them into the 64-bit run totals before any lane's segments pass 2^30
  unsigned n_launch = 0, n_flight = 0, n_coll = 0, n_seg = 0, n_esc = 0, n_rrk = 0, n_rrs = 0, n_scl = 0, n_evl = 0;
  double w_launch = 0.0, w_esc = 0.0, w_rr = 0.0, w_kill = 0.0;
  auto flush_counts = [&]() {
    DevStats *s = p.stats;
    unsigned long long evl = 0;
    auto put = [&](unsigned long long *dst, unsigned &v) {
      const unsigned long long t = wsum((unsigned long long)v);
      if (lane == 0 && t) atomicAdd(dst, t);
      v = 0;
      return t;
    };
    auto putw = [&](double *dst, double &v) {
      const double t = wsum(v);
      if (lane == 0) atomicAdd(dst, t);
      v = 0.0;
    };
    put(&s->launched, n_launch);
    put(&s->flights, n_flight);
    put(&s->collisions, n_coll);
    put(&s->segments, n_seg);
    put(&s->escapes, n_esc);
    put(&s->rr_kill, n_rrk);
    put(&s->rr_survive, n_rrs);
    put(&s->scatter_limit, n_scl);
    evl = put(&s->event_limit, n_evl);
    putw(&s->launched_w, w_launch);
    putw(&s->escaped_w, w_esc);
    putw(&s->rr_net_w, w_rr);
    putw(&s->killed_w, w_kill);
    if (lane == 0 && evl) atomicOr(p.flags, kFlagEventLimit);
  };

  // a new free flight (event flight + 1): tau = -ln U, the scattering uniforms, and the harmonics
  // of the direction; false when the event cap ends the packet first
  auto begin_flight = [&]() -> bool {
    if (flight >= p.max_events) {
      ++n_evl;
      w_kill += W;
      return false;
    }
    ++flight;
    ++n_flight;
    const uint4 r = philox4x32_10(pid, flight + 1u, p.key0, p.key1);
    tau = -logf(u01(r.x));
    cu1 = r.y;
    cu2 = r.z;
    cu3 = r.w;
    inv_ax = __frcp_rn(fabsf(ux));
    inv_ay = __frcp_rn(fabsf(uy));
    inv_az = __frcp_rn(fabsf(uz));
    if (MERGE) rb ^= 1;
    sh_row(p, ux, uy, uz, myrows + rb * p.row_stride);
    return true;
  };

  for (;;) {
    // ------------------------------------------------------------- refill
    const unsigned need = __ballot_sync(kFull3, !alive && !exhausted);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(p.work, (unsigned long long)__popc(need));
      base = __shfl_sync(kFull3, base, leader);
      if (!alive && !exhausted) {
        const unsigned long long g = base + __popc(need & ((1u << lane) - 1u));
        if (g >= p.n_packets) {
          exhausted = true;
        } else {
          pid = p.first_packet + g;
          ++n_launch;
          const uint4 r0 = philox4x32_10(pid, 0u, p.key0, p.key1);
          float x = p.x0, y = p.y0, z = p.z0;
          int vx = -1, vy = 0, vz = 0;
          W0 = 1.f;
          if (p.kind < 0) {  // volumetric: voxel by |q|, uniform in it, W0 = sign q
            const unsigned long long total = __ldg(p.cdf + nvox - 1);
            if (total == 0ull) {  // all-zero source: nothing to launch
              W0 = 0.f;
              x = -1.f;
            } else {
              const int v = pick_voxel(p.cdf, nvox, total, r0.x, r0.y);
              const uint4 r1 = philox4x32_10(pid, 1u, p.key0, p.key1);
              vx = v % p.nx;
              vy = (v / p.nx) % p.ny;
              vz = v / (p.nx * p.ny);
              x = u01(r1.x) * dx;
              y = u01(r1.y) * dx;
              z = u01(r1.z) * dx;
              W0 = __ldg(p.q + v) < 0.f ? -1.f : 1.f;
            }
          }
          if (p.kind == MCR_PENCIL) {
            ux = p.ux0;
            uy = p.uy0;
            uz = p.uz0;
          } else {  // isotropic: cos th = 2u - 1, ph = 2 pi u'
            const float ct = 2.f * u01(r0.z) - 1.f, st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
            float sp, cp;
            sincospif(2.f * u01(r0.w), &sp, &cp);
            ux = st * cp;
            uy = st * sp;
            uz = ct;
          }
          W = W0;
          w_launch += W0;
          flight = 0;
          nscat = 0;
          const bool inside =
              vx >= 0 || (x >= 0.f && x <= p.nx * dx && y >= 0.f && y <= p.ny * dx && z >= 0.f && z <= p.nz * dx);
          if (!inside) {
            ++n_esc;
            w_esc += W;
          } else {
            if (vx >= 0) {  // (x, y, z) already the offsets in voxel (vx, vy, vz)
              ix = vx;
              iy = vy;
              iz = vz;
              fx = x;
              fy = y;
              fz = z;
            } else {
              ix = min((int)floorf(x / dx), p.nx - 1);
              iy = min((int)floorf(y / dx), p.ny - 1);
              iz = min((int)floorf(z / dx), p.nz - 1);
              fx = clamp3(x - ix * dx, dx);
              fy = clamp3(y - iy * dx, dx);
              fz = clamp3(z - iz * dx, dx);
            }
            alive = begin_flight();
          }
        }
      }
    }
    if (!__any_sync(kFull3, alive)) break;
    __syncwarp();

    // ------------------------------------------------------------- one voxel segment
    int seg_v = -1;
    float seg_ts = 0.f, seg_carry = 0.f;
    bool collided = false, escaped = false;
    if (alive) {
      const int v = (iz * p.ny + iy) * p.nx + ix;
      const float4 m = __ldg(p.mu + v);
      const float dxf = ux != 0.f ? (ux > 0.f ? dx - fx : fx) * inv_ax : CUDART_INF_F;
      const float dyf = uy != 0.f ? (uy > 0.f ? dx - fy : fy) * inv_ay : CUDART_INF_F;
      const float dzf = uz != 0.f ? (uz > 0.f ? dx - fz : fz) * inv_az : CUDART_INF_F;
      int axis = 0;  // ties: x first, then y, then z
      float d_face = dxf;
      if (dyf < d_face) {
        d_face = dyf;
        axis = 1;
      }
      if (dzf < d_face) {
        d_face = dzf;
        axis = 2;
      }
      d_face = fmaxf(d_face, 0.f);
      const float d_coll = tau * m.w;  // +inf when mu_s = 0
      collided = d_coll < d_face;
      const float l = collided ? d_coll : d_face;
      const float em1 = expm1f(-m.x * l);
      const float t = m.x > 0.f ? (-W * em1) * m.z : W * l;
      W = fmaf(W, em1, W);
      ++n_seg;
      if (MERGE) {
        seg_carry = carry;
        carry = 0.f;
      }
      if (t != 0.f || seg_carry != 0.f) {
        seg_v = v;
        seg_ts = t * p.qscale;
      }
      if (MERGE && collided && t != 0.f && seg_carry == 0.f) {
        // defer it if the packet survives the collision (the tests below, in their order): its
        // next segment starts in this voxel
        const bool dies = nscat >= p.max_scatter ||
                          (fabsf(W) < p.w_threshold * fabsf(W0) && !(u01(cu2) < p.rr_p)) || flight >= p.max_events;
        if (!dies) {
          carry = seg_ts;
          seg_v = -1;
        }
      }
      // advance along the path; a face crossing then steps the voxel index on its axis and puts
      // the offset on the entered face (selects, not branches: the lanes of a warp take
      // different axes)
      fx = clamp3(fmaf(l, ux, fx), dx);
      fy = clamp3(fmaf(l, uy, fy), dx);
      fz = clamp3(fmaf(l, uz, fz), dx);
      if (!collided) {
        tau = fmaxf(fmaf(-m.y, l, tau), 0.f);
        const bool cx = axis == 0, cy = axis == 1, cz = axis == 2;
        ix += cx ? (ux > 0.f ? 1 : -1) : 0;
        iy += cy ? (uy > 0.f ? 1 : -1) : 0;
        iz += cz ? (uz > 0.f ? 1 : -1) : 0;
        fx = cx ? (ux > 0.f ? 0.f : dx) : fx;
        fy = cy ? (uy > 0.f ? 0.f : dx) : fy;
        fz = cz ? (uz > 0.f ? 0.f : dx) : fz;
        escaped = (unsigned)ix >= (unsigned)p.nx || (unsigned)iy >= (unsigned)p.ny || (unsigned)iz >= (unsigned)p.nz;
      }
    }

    // ------------------------------------------------------------- cooperative deposit
    unsigned pend = __ballot_sync(kFull3, seg_v >= 0);
    while (pend) {
      const int L = __ffs(pend) - 1;
      pend &= pend - 1u;
      const int v = __shfl_sync(kFull3, seg_v, L);
      const float ts = __shfl_sync(kFull3, seg_ts, L);
      unsigned long long *dst = p.tally + (size_t)v * p.Cpad;
      if (MERGE) {
        const float tc = __shfl_sync(kFull3, seg_carry, L);
        const int rbl = __shfl_sync(kFull3, rb, L);
        const float *row = warprows + (size_t)(2 * L + rbl) * p.row_stride;
        const float *prev = warprows + (size_t)(2 * L + (rbl ^ 1)) * p.row_stride;
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
          const int j = k * 32 + lane;
          if (j < p.C) {
            long long q = __float2int_rn(ts * row[j]);
            if (tc != 0.f) q += __float2int_rn(tc * prev[j]);
            atomicAdd(dst + j, (unsigned long long)q);
          }
        }
      } else {
        const float *row = warprows + (size_t)L * p.row_stride;
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
          const int j = k * 32 + lane;
          if (j < p.C) atomicAdd(dst + j, (unsigned long long)(long long)__float2int_rn(ts * row[j]));
        }
      }
    }
    __syncwarp();

    // ------------------------------------------------------------- escape / collision
    if (alive) {
      if (escaped) {
        ++n_esc;
        w_esc += W;
        alive = false;
      } else if (collided) {
        ++n_coll;
        if (nscat >= p.max_scatter) {
          ++n_scl;
          w_kill += W;
          alive = false;
        } else {
          turn(ux, uy, uz, hg3_cos(p.g, u01(cu1)), u01(cu3));
          ++nscat;
          if (fabsf(W) < p.w_threshold * fabsf(W0)) {
            if (u01(cu2) < p.rr_p) {
              const float Wn = W * p.rr_inv_p;
              ++n_rrs;
              w_rr += (double)Wn - (double)W;
              W = Wn;
            } else {
              ++n_rrk;
              w_rr -= W;
              alive = false;
            }
          }
          if (alive) alive = begin_flight();
        }
      }
    }
    if (__any_sync(kFull3, n_seg > (1u << 30))) flush_counts();
  }
  flush_counts();
}

// coeff[c][v] (+)= sum * quantum * scale, (-1)^l on odd l when adjoint; scale = fixed_scale or, for
// a volumetric source, 4 pi qmax total 2^-32 / N_p (S / (N_p V) with S = 4 pi V qmax total 2^-32)
__global__ void k_finalize3(const unsigned long long *__restrict__ tally, int64_t nvox, int C, int Cpad,
                            double quantum, double fixed_scale, int volumetric, const unsigned *qmax_bits,
                            const unsigned long long *cdf_total, double n_packets, int adjoint, int accumulate,
                            float *__restrict__ coeff, unsigned *flags) {
  double scale = fixed_scale;
  if (volumetric)
    scale = 4.0 * CUDART_PI * (double)__uint_as_float(*qmax_bits) * (double)(*cdf_total) * (1.0 / 4294967296.0) /
            n_packets;
  bool near = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvox * C; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / nvox);
    const int64_t v = i - (int64_t)c * nvox;
    const long long s = (long long)tally[v * Cpad + c];
    near |= (s > (1ll << 61)) || (s < -(1ll << 61));
    int l = 0;
    while ((l + 1) * (l + 1) <= c) ++l;
    const double sgn = (adjoint && (l & 1)) ? -1.0 : 1.0;
    const float val = (float)(sgn * (double)s * quantum * scale);
    coeff[i] = accumulate ? coeff[i] + val : val;
  }
  if (near) atomicOr(flags, kFlagOverflow);
}

// H = mu_a sqrt(4 pi) c_00; r = Hmeas - H; dL/dH = -V r; per-block FP64 sums of r^2
__global__ void k_h_eps3(const float *mua, const float *c00, const float *Hm, int64_t n, double V, float *H,
                         float *dLdH, double *partials) {
  __shared__ double red[256 / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float h = mua[i] * (float)(sqrt(4.0 * CUDART_PI) * (double)c00[i]);
    H[i] = h;
    if (Hm) {
      const double r = (double)Hm[i] - (double)h;
      if (dLdH) dLdH[i] = (float)(-V * r);
      acc += r * r;
    }
  }
  if (!partials) return;
  acc = wsum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

__global__ void k_eps3_final(const double *partials, int n, double half_V, double *eps) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += partials[i];
  *eps = half_V * s;
}

// d_mua = v sqrt(4 pi) c_00 + V sum_c c c*, d_mus = V sum_c (1 - g^l) c c* (FP64, increasing c);
// OUT double, or float (the FP64 result rounded once)
template <typename OUT>
__global__ void k_gradient3(const float *__restrict__ co, const float *__restrict__ ca, const float *__restrict__ v,
                            int64_t n, int C, double g, double V, OUT *d_mua, OUT *d_mus) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double sa = 0.0, ss = 0.0, gl = 1.0;
    int l = 0;
    for (int c = 0; c < C; ++c) {
      if ((l + 1) * (l + 1) <= c) {
        ++l;
        gl *= g;
      }
      const double p = (double)co[(int64_t)c * n + i] * (double)ca[(int64_t)c * n + i];
      sa += p;
      ss += (1.0 - gl) * p;
    }
    d_mua[i] = (OUT)((double)v[i] * sqrt(4.0 * CUDART_PI) * (double)co[i] + V * sa);
    d_mus[i] = (OUT)(V * ss);
  }
}

// -------------------------------------------------------------------- host side
struct Work3 {
  unsigned long long *tally = nullptr;
  size_t tally_bytes = 0;
  unsigned long long *cdf = nullptr, *block_sums = nullptr;
  size_t cdf_bytes = 0, bs_bytes = 0;
  float4 *mu = nullptr;
  size_t mu_bytes = 0;
  unsigned char *small = nullptr;  // [0,8) counter, [64,192) stats, [448] flags, [512] qmax bits
  double *partials = nullptr;
};
std::mutex g_mu3;
Work3 g_w3[64];

// Words per voxel row: above 16 channels whole 128-byte lines (each deposit then touches the
// fewest lines; rows of 28 words for 25 channels reduced 30 % slower from HBM than rows of 32),
// else a multiple of 4 (32-byte sectors).
int tally_row_words3(int C) { return C > 16 ? (C + 15) & ~15 : (C + 3) & ~3; }

int grow3(void **p, size_t *have, size_t need) {
  if (need <= *have) return MCR_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need) != cudaSuccess) return MCR_ERR_NOMEM;
  *have = need;
  return MCR_OK;
}

int work3(size_t tally, size_t nvox, Work3 **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MCR_ERR_CUDA;
  Work3 &w = g_w3[dev];
  int rc;
  if (!w.small) {
    if (cudaMalloc(&w.small, 1024) != cudaSuccess) return MCR_ERR_NOMEM;
    if (cudaMemset(w.small, 0, 1024) != cudaSuccess) return MCR_ERR_CUDA;
    if (cudaMalloc(&w.partials, 4096 * sizeof(double)) != cudaSuccess) return MCR_ERR_NOMEM;
  }
  if ((rc = grow3((void **)&w.tally, &w.tally_bytes, tally))) return rc;
  if ((rc = grow3((void **)&w.cdf, &w.cdf_bytes, nvox * 8))) return rc;
  if ((rc = grow3((void **)&w.mu, &w.mu_bytes, nvox * sizeof(float4)))) return rc;
  if ((rc = grow3((void **)&w.block_sums, &w.bs_bytes, ((nvox + 255) / 256) * 8))) return rc;
  *out = &w;
  return MCR_OK;
}

#define MCR3_TRY(expr)                          \
  do {                                          \
    if ((expr) != cudaSuccess) return MCR_ERR_CUDA; \
  } while (0)

int check_medium3(const mcr3_medium *m) {
  if (!m || !m->mua || !m->mus) return MCR_ERR_ARG;
  if (m->nx <= 0 || m->ny <= 0 || m->nz <= 0) return MCR_ERR_ARG;
  if ((int64_t)m->nx * m->ny * m->nz >= ((int64_t)1 << 26)) return MCR_ERR_ARG;
  if (!(m->dx > 0.f) || !isfinite(m->dx) || !(m->g > -1.f && m->g < 1.f)) return MCR_ERR_ARG;
  return MCR_OK;
}

int run3(const mcr3_medium *med, const mcr3_source *src, const float *qstar, const mcr_run *run, float *coeff,
         mcr_stats *stats, cudaStream_t s) {
  int rc;
  if ((rc = check_medium3(med))) return rc;
  if (!run || !coeff) return MCR_ERR_ARG;
  if (run->K < 0 || run->K > MCR3_MAX_L || run->sectors || run->time_bins || run->accumulate > 1u) return MCR_ERR_ARG;
  if (!(run->roulette_p > 0.f && run->roulette_p <= 1.f) || !(run->w_threshold >= 0.f)) return MCR_ERR_ARG;
  if (run->n_packets > (1ull << 26) || run->first_packet + run->n_packets < run->first_packet) return MCR_ERR_ARG;
  Transport3Params p;
  memset(&p, 0, sizeof(p));
  if (!qstar) {
    if (!src || (src->kind != MCR_PENCIL && src->kind != MCR_ISO_POINT)) return MCR_ERR_ARG;
    if (!isfinite(src->x0) || !isfinite(src->y0) || !isfinite(src->z0) || !isfinite(src->power)) return MCR_ERR_ARG;
    p.kind = src->kind;
    p.x0 = src->x0;
    p.y0 = src->y0;
    p.z0 = src->z0;
    if (src->kind == MCR_PENCIL) {
      const double n = sqrt((double)src->dir_x * src->dir_x + (double)src->dir_y * src->dir_y +
                            (double)src->dir_z * src->dir_z);
      if (!(n > 0.0) || !isfinite(n)) return MCR_ERR_ARG;
      p.ux0 = (float)(src->dir_x / n);
      p.uy0 = (float)(src->dir_y / n);
      p.uz0 = (float)(src->dir_z / n);
    }
  } else {
    p.kind = -1;
  }
  const int L = run->K, C = (L + 1) * (L + 1), Cpad = tally_row_words3(C);
  const int64_t nvox = (int64_t)med->nx * med->ny * med->nz;
  std::lock_guard<std::mutex> lock(g_mu3);
  Work3 *w = nullptr;
  if ((rc = work3((size_t)nvox * Cpad * 8, (size_t)nvox, &w))) return rc;
  unsigned long long *counter = reinterpret_cast<unsigned long long *>(w->small);
  DevStats *dstats = reinterpret_cast<DevStats *>(w->small + 64);
  unsigned *flags = reinterpret_cast<unsigned *>(w->small + 448);
  unsigned *qmax = reinterpret_cast<unsigned *>(w->small + 512);
  MCR3_TRY(cudaMemsetAsync(w->small, 0, 512, s));  // counter, stats, flags
  MCR3_TRY(cudaMemsetAsync(w->tally, 0, (size_t)nvox * Cpad * 8, s));
  MCR3_TRY(launch_pack_medium(med->mua, med->mus, w->mu, nvox, flags, s));
  if (qstar) MCR3_TRY(launch_source_cdf(qstar, nvox, w->cdf, w->block_sums, (size_t)((nvox + 255) / 256), qmax, s));
  p.nx = med->nx;
  p.ny = med->ny;
  p.nz = med->nz;
  p.dx = med->dx;
  p.g = med->g;
  p.L = L;
  p.C = C;
  p.Cpad = Cpad;
  p.row_stride = C | 1;  // odd: the lanes' rows fall in distinct banks
  p.mu = w->mu;
  p.tally = w->tally;
  p.cdf = w->cdf;
  p.q = qstar;
  p.key0 = (unsigned)run->seed;
  p.key1 = (unsigned)(run->seed >> 32) ^ run->stream_id;
  p.first_packet = run->first_packet;
  p.n_packets = run->n_packets;
  p.max_scatter = run->max_scatter;
  p.max_events = run->max_events;
  p.w_threshold = run->w_threshold;
  p.rr_p = run->roulette_p;
  p.rr_inv_p = 1.f / run->roulette_p;
  // q: every deposit |t Y_lm| 2^q < 2^30: t <= W l, l <= dx sqrt 3 in a voxel, |W| <= max(1,
  // w_threshold / p), |Y_lm| <= sqrt((2L+1) / 4 pi) (their squares over m sum to that)
  const double wmax = fmax(1.0, (double)run->w_threshold / (double)run->roulette_p);
  const double ymax = fmax(1.0, sqrt((2.0 * L + 1.0) / (4.0 * M_PI)));
  int qe = (int)floor(30.0 - log2(wmax * (double)med->dx * sqrt(3.0) * ymax * 1.001));
  qe = qe > 60 ? 60 : (qe < -60 ? -60 : qe);
  p.qscale = ldexpf(1.f, qe);
  for (int k = 1; k <= MCR3_MAX_L; ++k) p.rinv[k] = 1.f / (float)k;
  for (int l = 0; l <= L; ++l)
    for (int m = 0; m <= l; ++m) {
      double ratio = 1.0;
      for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
      const double N = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * ratio) * (m ? M_SQRT2 : 1.0);
      p.nlm[l * l + l + m] = (float)N;
    }
  p.work = counter;
  p.stats = dstats;
  p.flags = flags;
  if (run->n_packets) {
    int dev = 0, sms = 0, per_sm = 0;
    MCR3_TRY(cudaGetDevice(&dev));
    MCR3_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int nch = (C + 31) / 32;
    const bool merge = p.row_stride <= 25;  // two rows per lane still leave 8 blocks per SM
    const size_t smem = (size_t)kThreads3 * (merge ? 2 : 1) * p.row_stride * sizeof(float);
    if (merge) {
      MCR3_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_transport3<1, true>, kThreads3, smem));
      k_transport3<1, true><<<sms * (per_sm > 0 ? per_sm : 1), kThreads3, smem, s>>>(p);
    } else if (nch == 1) {
      MCR3_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_transport3<1, false>, kThreads3, smem));
      k_transport3<1, false><<<sms * (per_sm > 0 ? per_sm : 1), kThreads3, smem, s>>>(p);
    } else if (nch == 2) {
      MCR3_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_transport3<2, false>, kThreads3, smem));
      k_transport3<2, false><<<sms * (per_sm > 0 ? per_sm : 1), kThreads3, smem, s>>>(p);
    } else {
      MCR3_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_transport3<3, false>, kThreads3, smem));
      k_transport3<3, false><<<sms * (per_sm > 0 ? per_sm : 1), kThreads3, smem, s>>>(p);
    }
    MCR3_TRY(cudaGetLastError());
  }
  const double V = (double)med->dx * med->dx * med->dx;
  const double fixed = (!qstar && run->n_packets) ? (double)src->power / ((double)run->n_packets * V) : 0.0;
  k_finalize3<<<512, 256, 0, s>>>(w->tally, nvox, C, Cpad, ldexp(1.0, -qe), fixed, qstar && run->n_packets ? 1 : 0,
                                  qmax, w->cdf + (nvox - 1), (double)(run->n_packets ? run->n_packets : 1),
                                  qstar ? 1 : 0, run->accumulate ? 1 : 0, coeff, flags);
  MCR3_TRY(cudaGetLastError());
  DevStats d;
  unsigned f = 0;
  MCR3_TRY(cudaMemcpyAsync(&d, dstats, sizeof(d), cudaMemcpyDeviceToHost, s));
  MCR3_TRY(cudaMemcpyAsync(&f, flags, sizeof(f), cudaMemcpyDeviceToHost, s));
  MCR3_TRY(cudaStreamSynchronize(s));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->launched = d.launched;
    stats->flights = d.flights;
    stats->collisions = d.collisions;
    stats->segments = d.segments;
    stats->escapes = d.escapes;
    stats->rr_kill = d.rr_kill;
    stats->rr_survive = d.rr_survive;
    stats->scatter_limit = d.scatter_limit;
    stats->event_limit = d.event_limit;
    stats->launched_w = d.launched_w;
    stats->escaped_w = d.escaped_w;
    stats->rr_net_w = d.rr_net_w;
    stats->killed_w = d.killed_w;
    stats->absorbed_w = d.launched_w + d.rr_net_w - d.escaped_w - d.killed_w;
  }
  if (f & kFlagMedium) return MCR_ERR_MEDIUM;
  if (f & kFlagOverflow) return MCR_ERR_TALLY_OVERFLOW;
  if (f & kFlagEventLimit) return MCR_ERR_EVENT_LIMIT;
  return MCR_OK;
}

}  // namespace

// Frees this device's 3D workspace (called by mc_release_workspace).
int release_workspace3(int dev) {
  if (dev < 0 || dev >= 64) return MCR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu3);
  Work3 &w = g_w3[dev];
  void *ptrs[] = {w.tally, w.cdf, w.block_sums, w.mu, w.small, w.partials};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  w = Work3{};
  return MCR_OK;
}
}  // namespace mcr

using namespace mcr;

namespace {
template <typename OUT>
int gradient3(const mcr3_medium *med, int32_t L, const float *coeff, const float *coeff_adj, const float *dL_dH,
              OUT *d_mua, OUT *d_mus, void *stream) {
  int rc;
  if ((rc = check_medium3(med))) return rc;
  if (L < 0 || L > MCR3_MAX_L || !coeff || !coeff_adj || !dL_dH || !d_mua || !d_mus) return MCR_ERR_ARG;
  const int64_t n = (int64_t)med->nx * med->ny * med->nz;
  const double V = (double)med->dx * med->dx * med->dx;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_gradient3<OUT><<<grid, 256, 0, (cudaStream_t)stream>>>(coeff, coeff_adj, dL_dH, n, (L + 1) * (L + 1),
                                                            (double)med->g, V, d_mua, d_mus);
  return cudaGetLastError() == cudaSuccess ? MCR_OK : MCR_ERR_CUDA;
}

}  // namespace

extern "C" {

int mc3_forward(const mcr3_medium *med, const mcr3_source *src, const mcr_run *run, float *coeff, mcr_stats *stats,
                void *stream) {
  if (!src) return MCR_ERR_ARG;
  return run3(med, src, nullptr, run, coeff, stats, (cudaStream_t)stream);
}

int mc3_adjoint(const mcr3_medium *med, const float *qstar, const mcr_run *run, float *coeff_adj, mcr_stats *stats,
                void *stream) {
  if (!qstar) return MCR_ERR_ARG;
  return run3(med, nullptr, qstar, run, coeff_adj, stats, (cudaStream_t)stream);
}

int mc3_h_eps(const mcr3_medium *med, const float *coeff, const float *Hmeas, float *H, float *dL_dH, double *eps,
              void *stream) {
  int rc;
  if ((rc = check_medium3(med))) return rc;
  if (!coeff || !H) return MCR_ERR_ARG;
  const int64_t n = (int64_t)med->nx * med->ny * med->nz;
  const double V = (double)med->dx * med->dx * med->dx;
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_mu3);
  Work3 *w = nullptr;
  if ((rc = work3(0, 1, &w))) return rc;
  const int grid = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  k_h_eps3<<<grid, 256, 0, s>>>(med->mua, coeff, Hmeas, n, V, H, dL_dH, (Hmeas && eps) ? w->partials : nullptr);
  if (Hmeas && eps) k_eps3_final<<<1, 1, 0, s>>>(w->partials, grid, 0.5 * V, eps);
  return cudaGetLastError() == cudaSuccess ? MCR_OK : MCR_ERR_CUDA;
}

int mc3_adjoint_source(const mcr3_medium *med, const float *dL_dH, float *qstar, void *stream) {
  int rc;
  if ((rc = check_medium3(med))) return rc;
  if (!dL_dH || !qstar) return MCR_ERR_ARG;
  const int64_t n = (int64_t)med->nx * med->ny * med->nz;
  const double V = (double)med->dx * med->dx * med->dx;
  return launch_adjoint_source(med->mua, dL_dH, n, V, qstar, (cudaStream_t)stream) == cudaSuccess ? MCR_OK
                                                                                                   : MCR_ERR_CUDA;
}

int mc3_gradient(const mcr3_medium *med, int32_t L, const float *coeff, const float *coeff_adj, const float *dL_dH,
                 double *d_mua, double *d_mus, void *stream) {
  return gradient3(med, L, coeff, coeff_adj, dL_dH, d_mua, d_mus, stream);
}

int mc3_gradient_f32(const mcr3_medium *med, int32_t L, const float *coeff, const float *coeff_adj,
                     const float *dL_dH, float *d_mua, float *d_mus, void *stream) {
  return gradient3(med, L, coeff, coeff_adj, dL_dH, d_mua, d_mus, stream);
}

}  // extern "C"
