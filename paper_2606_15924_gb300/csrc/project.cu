// EWA projection with SH colour (the 3DGS forward model TurboGS rasterizes,
// Sec. 3.1) and its adjoint.  One thread per Gaussian; SH coefficients and
// quaternions move as float4; a Gaussian that misses every active tile is
// culled before its SH block is read.
#include "hybrid_math.cuh"

namespace tgs {

struct CamK {
  float W[9], t[3], campos[3];
  float fx, fy, cx, cy, znear, limx, limy;
  int width, height, tx, ty;
};

static CamK make_cam(const tgs_camera& c) {
  CamK k;
  for (int r = 0; r < 3; ++r) {
    for (int j = 0; j < 3; ++j) k.W[r * 3 + j] = c.viewmat[r * 4 + j];
    k.t[r] = c.viewmat[r * 4 + 3];
  }
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
    for (int r = 0; r < 3; ++r) s += (double)c.viewmat[r * 4 + j] * (double)c.viewmat[r * 4 + 3];
    k.campos[j] = (float)(-s);
  }
  k.fx = c.fx; k.fy = c.fy; k.cx = c.cx; k.cy = c.cy; k.znear = c.znear;
  k.limx = (float)(1.3 * (0.5 * c.width / (double)c.fx));
  k.limy = (float)(1.3 * (0.5 * c.height / (double)c.fy));
  k.width = c.width; k.height = c.height;
  k.tx = tiles_x(c.width); k.ty = tiles_y(c.height);
  return k;
}

// Real spherical harmonics of degree <= 3 (Condon-Shortley phase), m = -l..l
// ordered, as polynomials of the unit direction.
#define SH_C0 0.28209479177387814f
#define SH_C1 0.4886025119029199f
__constant__ float kSH2[5] = {1.0925484305920792f, -1.0925484305920792f, 0.31539156525252005f,
                              -1.0925484305920792f, 0.5462742152960396f};
__constant__ float kSH3[7] = {-0.5900435899266435f, 2.890611442640554f, -0.4570457994644658f,
                              0.3731763325901154f, -0.4570457994644658f, 1.445305721320277f,
                              -0.5900435899266435f};

__device__ __forceinline__ void sh_basis(float x, float y, float z, int deg, float Y[16]) {
  Y[0] = SH_C0;
  if (deg < 1) return;
  Y[1] = -SH_C1 * y; Y[2] = SH_C1 * z; Y[3] = -SH_C1 * x;
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kSH2[0] * x * y;
  Y[5] = kSH2[1] * y * z;
  Y[6] = kSH2[2] * (2.f * zz - xx - yy);
  Y[7] = kSH2[3] * x * z;
  Y[8] = kSH2[4] * (xx - yy);
  if (deg < 3) return;
  Y[9] = kSH3[0] * y * (3.f * xx - yy);
  Y[10] = kSH3[1] * x * y * z;
  Y[11] = kSH3[2] * y * (4.f * zz - xx - yy);
  Y[12] = kSH3[3] * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = kSH3[4] * x * (4.f * zz - xx - yy);
  Y[14] = kSH3[5] * z * (xx - yy);
  Y[15] = kSH3[6] * x * (xx - 3.f * yy);
}

// gradient of sum_k s_k Y_k with respect to the (unnormalised) polynomial argument
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, int deg, const float s[16], float g[3]) {
  g[0] = g[1] = g[2] = 0.f;
  if (deg < 1) return;
  g[0] += -SH_C1 * s[3]; g[1] += -SH_C1 * s[1]; g[2] += SH_C1 * s[2];
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  g[0] += kSH2[0] * y * s[4] + kSH2[3] * z * s[7] - 2.f * kSH2[2] * x * s[6] + 2.f * kSH2[4] * x * s[8];
  g[1] += kSH2[0] * x * s[4] + kSH2[1] * z * s[5] - 2.f * kSH2[2] * y * s[6] - 2.f * kSH2[4] * y * s[8];
  g[2] += kSH2[1] * y * s[5] + 4.f * kSH2[2] * z * s[6] + kSH2[3] * x * s[7];
  if (deg < 3) return;
  g[0] += kSH3[0] * 6.f * x * y * s[9] + kSH3[1] * y * z * s[10] - 2.f * kSH3[2] * x * y * s[11] -
          6.f * kSH3[3] * x * z * s[12] + kSH3[4] * (4.f * zz - 3.f * xx - yy) * s[13] +
          2.f * kSH3[5] * x * z * s[14] + kSH3[6] * (3.f * xx - 3.f * yy) * s[15];
  g[1] += kSH3[0] * (3.f * xx - 3.f * yy) * s[9] + kSH3[1] * x * z * s[10] +
          kSH3[2] * (4.f * zz - xx - 3.f * yy) * s[11] - 6.f * kSH3[3] * y * z * s[12] -
          2.f * kSH3[4] * x * y * s[13] - 2.f * kSH3[5] * y * z * s[14] - 6.f * kSH3[6] * x * y * s[15];
  g[2] += kSH3[1] * x * y * s[10] + 8.f * kSH3[2] * y * z * s[11] +
          kSH3[3] * (6.f * zz - 3.f * xx - 3.f * yy) * s[12] + 8.f * kSH3[4] * x * z * s[13] +
          kSH3[5] * (xx - yy) * s[14];
}

// Geometry of one Gaussian up to the conic (everything but colour).
struct Geo {
  float pc[3];
  float q[4], qnorm, R[9], s[3];
  float Sig[6];  // xx xy xz yy yz zz
  float T[6];    // J W, 2x3
  bool clampx, clampy;
  float A, B, C, det;
  float conic[3];
  int radius;
  float xy[2];
};

// Returns false when culled by depth or determinant.
__device__ __forceinline__ bool geometry(const CamK& cam, float3 mu, float3 ls, float4 qr, Geo& g) {
  g.pc[0] = cam.W[0] * mu.x + cam.W[1] * mu.y + cam.W[2] * mu.z + cam.t[0];
  g.pc[1] = cam.W[3] * mu.x + cam.W[4] * mu.y + cam.W[5] * mu.z + cam.t[1];
  g.pc[2] = cam.W[6] * mu.x + cam.W[7] * mu.y + cam.W[8] * mu.z + cam.t[2];
  const float z = g.pc[2];
  if (!(z > cam.znear)) return false;
  g.qnorm = sqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
  const float iq = 1.f / g.qnorm;
  const float w = qr.x * iq, x = qr.y * iq, y = qr.z * iq, zq = qr.w * iq;
  g.q[0] = w; g.q[1] = x; g.q[2] = y; g.q[3] = zq;
  float* R = g.R;
  R[0] = 1.f - 2.f * (y * y + zq * zq); R[1] = 2.f * (x * y - w * zq);       R[2] = 2.f * (x * zq + w * y);
  R[3] = 2.f * (x * y + w * zq);       R[4] = 1.f - 2.f * (x * x + zq * zq); R[5] = 2.f * (y * zq - w * x);
  R[6] = 2.f * (x * zq - w * y);       R[7] = 2.f * (y * zq + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
  g.s[0] = expf(ls.x); g.s[1] = expf(ls.y); g.s[2] = expf(ls.z);
  float M[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[r * 3 + c] = R[r * 3 + c] * g.s[c];
  g.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  g.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
  g.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
  g.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
  g.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
  g.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
  const float iz = 1.f / z;
  const float xz = g.pc[0] * iz, yz = g.pc[1] * iz;
  g.clampx = (xz < -cam.limx) || (xz > cam.limx);
  g.clampy = (yz < -cam.limy) || (yz > cam.limy);
  const float txz = fminf(fmaxf(xz, -cam.limx), cam.limx);
  const float tyz = fminf(fmaxf(yz, -cam.limy), cam.limy);
  const float J00 = cam.fx * iz, J02 = -cam.fx * txz * iz, J11 = cam.fy * iz, J12 = -cam.fy * tyz * iz;
  // T = J W
  g.T[0] = J00 * cam.W[0] + J02 * cam.W[6];
  g.T[1] = J00 * cam.W[1] + J02 * cam.W[7];
  g.T[2] = J00 * cam.W[2] + J02 * cam.W[8];
  g.T[3] = J11 * cam.W[3] + J12 * cam.W[6];
  g.T[4] = J11 * cam.W[4] + J12 * cam.W[7];
  g.T[5] = J11 * cam.W[5] + J12 * cam.W[8];
  const float* S = g.Sig;
  // U = T Sigma (2x3)
  float U0 = g.T[0] * S[0] + g.T[1] * S[1] + g.T[2] * S[2];
  float U1 = g.T[0] * S[1] + g.T[1] * S[3] + g.T[2] * S[4];
  float U2 = g.T[0] * S[2] + g.T[1] * S[4] + g.T[2] * S[5];
  float U3 = g.T[3] * S[0] + g.T[4] * S[1] + g.T[5] * S[2];
  float U4 = g.T[3] * S[1] + g.T[4] * S[3] + g.T[5] * S[4];
  float U5 = g.T[3] * S[2] + g.T[4] * S[4] + g.T[5] * S[5];
  g.A = U0 * g.T[0] + U1 * g.T[1] + U2 * g.T[2] + 0.3f;
  g.B = U0 * g.T[3] + U1 * g.T[4] + U2 * g.T[5];
  g.C = U3 * g.T[3] + U4 * g.T[4] + U5 * g.T[5] + 0.3f;
  g.det = g.A * g.C - g.B * g.B;
  if (!(g.det > 0.f)) return false;
  const float idet = 1.f / g.det;
  g.conic[0] = g.C * idet; g.conic[1] = -g.B * idet; g.conic[2] = g.A * idet;
  const float mid = 0.5f * (g.A + g.C);
  const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - g.det));
  g.radius = (int)ceilf(3.f * sqrtf(lam));
  g.xy[0] = cam.fx * g.pc[0] * iz + cam.cx;
  g.xy[1] = cam.fy * g.pc[1] * iz + cam.cy;
  return true;
}

// Tile rectangle non-empty and (with a mask) holding an active tile.
__device__ __forceinline__ bool touches_active(const CamK& cam, const float xy[2], int radius,
                                               const int32_t* __restrict__ tile_rank) {
  int x0, x1, y0, y1;
  tile_span(xy[0], radius, cam.tx, x0, x1);
  tile_span(xy[1], radius, cam.ty, y0, y1);
  if ((x1 - x0) * (y1 - y0) == 0) return false;
  if (!tile_rank) return true;
  for (int ty = y0; ty < y1; ++ty)
    for (int tx = x0; tx < x1; ++tx)
      if (__ldg(tile_rank + ty * cam.tx + tx) >= 0) return true;
  return false;
}

__global__ void __launch_bounds__(256) k_project(
    GeoC geo, const float4* __restrict__ sh, int64_t n, int sh_degree, CamK cam,
    const int32_t* __restrict__ tile_rank, float2* __restrict__ xy_out, float4* __restrict__ conic_out,
    float* __restrict__ rgb_out, float* __restrict__ depth_out, int32_t* __restrict__ radius_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float3 mu = geo.mean(i);
  float3 ls = geo.lsc(i);
  float4 qr = geo.quat(i);
  Geo g;
  bool vis = geometry(cam, mu, ls, qr, g) && touches_active(cam, g.xy, g.radius, tile_rank);
  if (!vis) {
    xy_out[i] = make_float2(0.f, 0.f);
    conic_out[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    rgb_out[3 * i] = 0.f; rgb_out[3 * i + 1] = 0.f; rgb_out[3 * i + 2] = 0.f;
    depth_out[i] = 0.f;
    radius_out[i] = 0;
    return;
  }
  // colour from SH in the viewing direction
  float dx = mu.x - cam.campos[0], dy = mu.y - cam.campos[1], dz = mu.z - cam.campos[2];
  float il = rsqrtf(dx * dx + dy * dy + dz * dz);
  dx *= il; dy *= il; dz *= il;
  float Y[16];
  sh_basis(dx, dy, dz, sh_degree, Y);
  const int nb = (sh_degree + 1) * (sh_degree + 1);
  const float4* shp = sh + 12 * i;
  // the whole row (48 floats at every degree) in one round of loads: a loop
  // that stops at the degree would wait for each load in turn
  float4 row[12];
#pragma unroll
  for (int k4 = 0; k4 < 12; ++k4) row[k4] = ldg_f4_now(shp + k4);
  float acc[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
  for (int k4 = 0; k4 < 12; ++k4) {
    const float e[4] = {row[k4].x, row[k4].y, row[k4].z, row[k4].w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = 4 * k4 + j;  // flat index k * 3 + c
      const int k = f / 3, c = f - 3 * k;
      if (k < nb) acc[c] += e[j] * Y[k];
    }
  }
  xy_out[i] = make_float2(g.xy[0], g.xy[1]);
  conic_out[i] = make_float4(g.conic[0], g.conic[1], g.conic[2], 1.f / (1.f + expf(-geo.opac(i))));
  rgb_out[3 * i] = fmaxf(acc[0], 0.f);
  rgb_out[3 * i + 1] = fmaxf(acc[1], 0.f);
  rgb_out[3 * i + 2] = fmaxf(acc[2], 0.f);
  depth_out[i] = g.pc[2];
  radius_out[i] = g.radius;
}

bool gaussians_ok(const tgs_gaussians* g);
bool camera_ok(const tgs_camera* c);

// Adjoint of the projection.  grad2d rows: (dx, dy, da, db | dc, do, dr, dg | db, -, -, -).

// SH-coefficient gradient accumulators of the multi-view adjoint: a
// shared-memory column of the thread block (keeps the register count, hence
// the occupancy, up).
struct SmemSh {
  float* base;  // element k at base[k * stride]
  int stride;
  bool fresh = false;  // set: add() stores (the first view, no zeroing pass)
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 48; ++k) base[k * stride] = 0.f;
  }
  __device__ __forceinline__ void add(int k, float x) { base[k * stride] = fresh ? x : base[k * stride] + x; }
  __device__ __forceinline__ float get(int k) const { return base[k * stride]; }
};

// One view only: each float4 of the SH gradient is stored (or added to the
// gradient array) as soon as it is complete, so nothing stays live.
struct DirectSh {
  float4* out;
  bool accumulate;
  float st[4];
  __device__ __forceinline__ void zero() {}
  __device__ __forceinline__ void add(int k, float x) {
    st[k & 3] = x;
    if ((k & 3) == 3) {
      float4 v = make_float4(st[0], st[1], st[2], st[3]);
      if (accumulate) {
        const float4 q = out[k >> 2];
        v = make_float4(q.x + v.x, q.y + v.y, q.z + v.z, q.w + v.w);
      }
      out[k >> 2] = v;
    }
  }
};

// Parameter-gradient accumulators of one Gaussian.
template <class Sh>
struct AdjAcc {
  float mu[3], ls[3], q[4], o;
  Sh sh;
};

__device__ __forceinline__ bool grad2d_nonzero(float4 ga, float4 gb, float4 gc) {
  return ga.x != 0.f || ga.y != 0.f || ga.z != 0.f || ga.w != 0.f || gb.x != 0.f || gb.y != 0.f || gb.z != 0.f ||
         gb.w != 0.f || gc.x != 0.f;
}

// The colour part of one view's adjoint: the SH coefficients' gradient
// (Sh::add, coefficient j = 3 k + c of basis function k, channel c), given
// the colour gradient (dr, dg, db) of the view's projected Gaussian, and the
// direction term of the mean's gradient, dmu.  rw (nullable): the DC colour
// gradient of this view goes to rw[10..12].
template <class Sh>
__device__ __forceinline__ void view_colour(const CamK& cam, float3 mu, const float4* __restrict__ shp,
                                            int sh_degree, float dr, float dg, float db, float* __restrict__ rw,
                                            Sh& shacc, float (&dmu)[3]) {
  const float drgb[3] = {dr, dg, db};
  float vx = mu.x - cam.campos[0], vy = mu.y - cam.campos[1], vz = mu.z - cam.campos[2];
  const float il = rsqrtf(vx * vx + vy * vy + vz * vz);
  const float dx = vx * il, dy = vy * il, dz = vz * il;
  float Y[16];
  sh_basis(dx, dy, dz, sh_degree, Y);
  const int nb = (sh_degree + 1) * (sh_degree + 1);
  // the SH block is read twice (colour before the clamp, then the direction
  // gradient) rather than held in registers; the second read hits L1.
  // Coefficient j = 3 k + c belongs to basis function k, channel c; only
  // j < 3 nb exist at this degree (the rest of the gradient is zero).
  // loads in groups of four float4 issued together (a loop that stops at the
  // degree would wait for each load in turn); the row has 48 floats at every
  // degree
  float pre[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
  for (int g4 = 0; g4 < 12; g4 += 4) {
    float4 q[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) q[r] = shp[g4 + r];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float e[4] = {q[r].x, q[r].y, q[r].z, q[r].w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = 4 * (g4 + r) + u;
        if (j < 3 * nb) pre[j % 3] += e[u] * Y[j / 3];
      }
    }
  }
  const float dc0 = pre[0] >= 0.f ? drgb[0] : 0.f;
  const float dc1 = pre[1] >= 0.f ? drgb[1] : 0.f;
  const float dc2 = pre[2] >= 0.f ? drgb[2] : 0.f;
  const float dcv[3] = {dc0, dc1, dc2};
  float sk[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) sk[k] = 0.f;
  // an opaque copy of the row pointer: the compiler may not keep the first
  // pass's 48 values live in registers for this pass
  const float4* shp2 = shp;
  asm volatile("" : "+l"(shp2));
#pragma unroll
  for (int g4 = 0; g4 < 12; g4 += 4) {
    float4 q[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) q[r] = shp2[g4 + r];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float e[4] = {q[r].x, q[r].y, q[r].z, q[r].w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = 4 * (g4 + r) + u;
        const bool on = j < 3 * nb;
        if (on) sk[j / 3] += dcv[j % 3] * e[u];
        shacc.add(j, on ? dcv[j % 3] * Y[j / 3] : 0.f);
      }
    }
  }
  if (rw) {
    rw[10] = dc0 * Y[0];
    rw[11] = dc1 * Y[0];
    rw[12] = dc2 * Y[0];
  }
  float gd[3];
  sh_basis_grad(dx, dy, dz, sh_degree, sk, gd);
  const float dot = gd[0] * dx + gd[1] * dy + gd[2] * dz;
  dmu[0] = (gd[0] - dx * dot) * il;
  dmu[1] = (gd[1] - dy * dot) * il;
  dmu[2] = (gd[2] - dz * dot) * il;
}

// The geometry part of one view's adjoint, given the gradient (d_x, d_y) of
// the projected centre and (d_a, d_b, d_c) of the conic: the screen-space
// term of the mean's gradient dmu, and the gradients of the log-scales dls
// and the raw quaternion dq.
__device__ __forceinline__ void view_geometry(const CamK& cam, float3 mu, float3 ls, float4 qr, float d_x,
                                              float d_y, float d_a, float d_b, float d_c, float (&dmu)[3],
                                              float (&dls)[3], float (&dq4)[4]) {
  Geo g;
  geometry(cam, mu, ls, qr, g);  // visible by construction (radius > 0)
  // centre
  const float z = g.pc[2], iz = 1.f / z, iz2 = iz * iz;
  float dpc[3];
  dpc[0] = d_x * cam.fx * iz;
  dpc[1] = d_y * cam.fy * iz;
  dpc[2] = -d_x * cam.fx * g.pc[0] * iz2 - d_y * cam.fy * g.pc[1] * iz2;
  // conic Q = Sigma2^-1: dSigma2 = -Q dQ Q, dQ symmetric with off-diagonal db/2
  const float qa = g.conic[0], qb = g.conic[1], qc = g.conic[2];
  const float hb = 0.5f * d_b;
  // P = Q dQ
  const float P00 = qa * d_a + qb * hb, P01 = qa * hb + qb * d_c;
  const float P10 = qb * d_a + qc * hb, P11 = qb * hb + qc * d_c;
  // dS2 = -(P Q)
  const float S00 = -(P00 * qa + P01 * qb), S01 = -(P00 * qb + P01 * qc);
  const float S10 = -(P10 * qa + P11 * qb), S11 = -(P10 * qb + P11 * qc);
  const float Sym01 = 0.5f * (S01 + S10);
  // dSigma = T^T dS2 T (3x3 symmetric)
  const float* T = g.T;
  float dSig[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      dSig[r * 3 + c] = T[r] * (S00 * T[c] + Sym01 * T[3 + c]) + T[3 + r] * (Sym01 * T[c] + S11 * T[3 + c]);
  // dT = 2 dS2 T Sigma
  const float* Sg = g.Sig;
  const float Sfull[9] = {Sg[0], Sg[1], Sg[2], Sg[1], Sg[3], Sg[4], Sg[2], Sg[4], Sg[5]};
  float TS[6];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      TS[r * 3 + c] = T[r * 3] * Sfull[c] + T[r * 3 + 1] * Sfull[3 + c] + T[r * 3 + 2] * Sfull[6 + c];
  float dT[6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dT[c] = 2.f * (S00 * TS[c] + Sym01 * TS[3 + c]);
    dT[3 + c] = 2.f * (Sym01 * TS[c] + S11 * TS[3 + c]);
  }
  // dJ = dT W^T
  const float* Wm = cam.W;
  const float dJ00 = dT[0] * Wm[0] + dT[1] * Wm[1] + dT[2] * Wm[2];
  const float dJ02 = dT[0] * Wm[6] + dT[1] * Wm[7] + dT[2] * Wm[8];
  const float dJ11 = dT[3] * Wm[3] + dT[4] * Wm[4] + dT[5] * Wm[5];
  const float dJ12 = dT[3] * Wm[6] + dT[4] * Wm[7] + dT[5] * Wm[8];
  dpc[2] += dJ00 * (-cam.fx * iz2) + dJ11 * (-cam.fy * iz2);
  if (!g.clampx) {
    dpc[0] += dJ02 * (-cam.fx * iz2);
    dpc[2] += dJ02 * (2.f * cam.fx * g.pc[0] * iz2 * iz);
  } else {
    const float lim = g.pc[0] > 0.f ? cam.limx : -cam.limx;
    dpc[2] += dJ02 * (cam.fx * lim * iz2);
  }
  if (!g.clampy) {
    dpc[1] += dJ12 * (-cam.fy * iz2);
    dpc[2] += dJ12 * (2.f * cam.fy * g.pc[1] * iz2 * iz);
  } else {
    const float lim = g.pc[1] > 0.f ? cam.limy : -cam.limy;
    dpc[2] += dJ12 * (cam.fy * lim * iz2);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) dmu[a] = Wm[a] * dpc[0] + Wm[3 + a] * dpc[1] + Wm[6 + a] * dpc[2];
  // Sigma = M M^T, M = R diag(s): dM = 2 dSigma M
  const float* R = g.R;
  float M[9], dM[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[r * 3 + c] = R[r * 3 + c] * g.s[c];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      dM[r * 3 + c] = 2.f * (dSig[r * 3] * M[c] + dSig[r * 3 + 1] * M[3 + c] + dSig[r * 3 + 2] * M[6 + c]);
  float dR[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float ds = R[c] * dM[c] + R[3 + c] * dM[3 + c] + R[6 + c] * dM[6 + c];
    dls[c] = ds * g.s[c];
#pragma unroll
    for (int r = 0; r < 3; ++r) dR[r * 3 + c] = dM[r * 3 + c] * g.s[c];
  }
  const float w = g.q[0], x = g.q[1], y = g.q[2], zq = g.q[3];
  float dq[4];
  dq[0] = 2.f * (-zq * dR[1] + y * dR[2] + zq * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  dq[1] = 2.f * (y * dR[1] + zq * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + zq * dR[6] + w * dR[7] -
                 2.f * x * dR[8]);
  dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + zq * dR[5] - w * dR[6] + zq * dR[7] -
                 2.f * y * dR[8]);
  dq[3] = 2.f * (-2.f * zq * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * zq * dR[4] + y * dR[5] +
                 x * dR[6] + y * dR[7]);
  const float qd = dq[0] * w + dq[1] * x + dq[2] * y + dq[3] * zq;
  const float iq = 1.f / g.qnorm;
  const float gq[4] = {(dq[0] - w * qd) * iq, (dq[1] - x * qd) * iq, (dq[2] - y * qd) * iq, (dq[3] - zq * qd) * iq};
#pragma unroll
  for (int a = 0; a < 4; ++a) dq4[a] = gq[a];
}


// Adds one view's adjoint of the projection of Gaussian (mu, ls, qr, opacity
// o, SH block shp) into acc; rw (nullable) receives this view's own gradient
// row (means, log-scales, quaternion, DC r g b, opacity logit).
template <class Sh>
__device__ __forceinline__ void view_adjoint(const CamK& cam, float3 mu, float3 ls, float4 qr, float o,
                                             const float4* __restrict__ shp, int sh_degree, float4 ga, float4 gb,
                                             float4 gc, float* __restrict__ rw, AdjAcc<Sh>& acc) {
  const float g_o = gb.y * o * (1.f - o);
  acc.o += g_o;
  if (rw) rw[13] = g_o;
  float dmu_c[3];
  view_colour(cam, mu, shp, sh_degree, gb.z, gb.w, gc.x, rw, acc.sh, dmu_c);
  // the geometry after the colour part, so that its state and the SH basis
  // are not live at the same time
  float dmu_g[3], dls[3], dq[4];
  view_geometry(cam, mu, ls, qr, ga.x, ga.y, ga.z, ga.w, gb.x, dmu_g, dls, dq);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float d = dmu_c[a] + dmu_g[a];
    acc.mu[a] += d;
    if (rw) rw[a] = d;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc.ls[c] += dls[c];
    if (rw) rw[3 + c] = dls[c];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    acc.q[a] += dq[a];
    if (rw) rw[6 + a] = dq[a];
  }
}

template <class Sh>
__device__ __forceinline__ void acc_zero(AdjAcc<Sh>& a) {
#pragma unroll
  for (int k = 0; k < 3; ++k) a.mu[k] = a.ls[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) a.q[k] = 0.f;
  a.o = 0.f;
  a.sh.zero();
}

template <class Sh, class Put4>
__device__ __forceinline__ void store_sh(const Sh& sh, float4* out, Put4 put4) {
#pragma unroll
  for (int k4 = 0; k4 < 12; ++k4)
    put4(out + k4, make_float4(sh.get(4 * k4), sh.get(4 * k4 + 1), sh.get(4 * k4 + 2), sh.get(4 * k4 + 3)));
}
template <class Put4>
__device__ __forceinline__ void store_sh(const DirectSh&, float4*, Put4) {}  // stored as it was formed

// Writes (add = false) or adds (add = true) acc into the gradient arrays.
template <class Sh>
__device__ __forceinline__ void acc_store(const AdjAcc<Sh>& a, int64_t i, bool add, const GeoW& gw,
                                          float4* __restrict__ g_sh) {
  auto put = [&](float* p, float v) { *p = add ? *p + v : v; };
  auto put4 = [&](float4* p, float4 v) {
    if (add) {
      const float4 q = *p;
      v = make_float4(q.x + v.x, q.y + v.y, q.z + v.z, q.w + v.w);
    }
    *p = v;
  };
  float* gm = gw.mean(i);
  float* gl = gw.lsc(i);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    put(gm + k, a.mu[k]);
    put(gl + k, a.ls[k]);
  }
  put4(gw.quat(i), make_float4(a.q[0], a.q[1], a.q[2], a.q[3]));
  put(gw.opac(i), a.o);
  store_sh(a.sh, g_sh + 12 * i, put4);
}

__device__ __forceinline__ void zero_row(float* row, int64_t i) {
  float2* r2 = reinterpret_cast<float2*>(row + 14 * i);
#pragma unroll
  for (int k = 0; k < 7; ++k) r2[k] = make_float2(0.f, 0.f);
}

__device__ __forceinline__ void zero_grads(int64_t i, const GeoW& gw, float4* __restrict__ g_sh) {
  float* gm = gw.mean(i);
  float* gl = gw.lsc(i);
  gm[0] = 0.f; gm[1] = 0.f; gm[2] = 0.f;
  gl[0] = 0.f; gl[1] = 0.f; gl[2] = 0.f;
  *gw.quat(i) = make_float4(0.f, 0.f, 0.f, 0.f);
  *gw.opac(i) = 0.f;
#pragma unroll
  for (int k = 0; k < 12; ++k) g_sh[12 * i + k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void __launch_bounds__(256) k_project_bwd(
    GeoC geo, const float4* __restrict__ sh, int64_t n, int sh_degree, CamK cam,
    const int32_t* __restrict__ radius, const float4* __restrict__ grad2d, GeoW gw, float4* __restrict__ g_sh,
    uint8_t* __restrict__ touched, int write_untouched, int accumulate, float* __restrict__ row) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga, gc = ga;
  const bool vis = radius[i] > 0;
  if (vis) {
    ga = grad2d[3 * i];
    gb = grad2d[3 * i + 1];
    gc = grad2d[3 * i + 2];
  }
  const bool any = vis && grad2d_nonzero(ga, gb, gc);
  // accumulate: add into the gradients of Gaussians some earlier view of the
  // same step already touched, overwrite the rest (touched is the flag)
  const bool add = accumulate && touched[i] != 0;
  if (touched) {
    if (!accumulate) touched[i] = any ? 1 : 0;
    else if (any) touched[i] = 1;
  }
  if (!any) {
    if (row) zero_row(row, i);
    if (write_untouched && !accumulate) zero_grads(i, gw, g_sh);
    return;
  }
  const float3 mu = geo.mean(i);
  const float3 ls = geo.lsc(i);
  const float o = 1.f / (1.f + expf(-geo.opac(i)));
  AdjAcc<DirectSh> acc;
  acc_zero(acc);
  acc.sh.out = g_sh + 12 * i;
  acc.sh.accumulate = add;
  view_adjoint(cam, mu, ls, geo.quat(i), o, sh + 12 * i, sh_degree, ga, gb, gc, row ? row + 14 * i : nullptr,
               acc);
  acc_store(acc, i, add, gw, g_sh);
}

void launch_project_bwd(const tgs_gaussians& g, const tgs_camera& cam, const int32_t* radius, const float* grad2d,
                        const tgs_param_ptrs& grads, uint8_t* touched, int write_untouched, int accumulate,
                        float* row, cudaStream_t s) {
  if (g.n <= 0) return;
  CamK k = make_cam(cam);
  int blocks = (int)((g.n + 255) / 256);
  k_project_bwd<<<blocks, 256, 0, s>>>(geo_of(g), reinterpret_cast<const float4*>(g.sh), g.n, g.sh_degree, k,
                                       radius, reinterpret_cast<const float4*>(grad2d), geo_of(grads),
                                       reinterpret_cast<float4*>(grads.sh), touched, write_untouched, accumulate, row);
}

// Several views of one step in one pass: each Gaussian's parameters are read
// once, the views that touched it add their adjoints in registers, and its
// gradients are written once.
constexpr int kMaxAdjViews = 16;
struct MultiAdj {
  int n_views;
  CamK cam[kMaxAdjViews];
  const int32_t* radius[kMaxAdjViews];
  const float4* grad2d[kMaxAdjViews];
  float* row[kMaxAdjViews];
};

// Pass 1 over every Gaussian: which views touched it (touched, zero rows of
// the others, zero gradients if asked), and a compact list of the touched
// ones with their view masks (order of the list is irrelevant: every entry is
// computed on its own).
__global__ void __launch_bounds__(256) k_adj_mark(int64_t n, MultiAdj mv, uint8_t* __restrict__ touched,
                                                  int write_untouched, GeoW gw, float4* __restrict__ g_sh,
                                                  uint2* __restrict__ list, int32_t* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;
  unsigned hit = 0;
  if (valid) {
    for (int v = 0; v < mv.n_views; ++v) {
      bool any = false;
      if (mv.radius[v][i] > 0) {
        const float4* gp = mv.grad2d[v] + 3 * i;
        any = grad2d_nonzero(gp[0], gp[1], gp[2]);
      }
      if (any) hit |= 1u << v;
      else if (mv.row[v]) zero_row(mv.row[v], i);
    }
    if (touched) touched[i] = hit ? 1 : 0;
    if (!hit && write_untouched) zero_grads(i, gw, g_sh);
  }
  const int64_t pos = block_append(hit != 0, count);
  if (hit) list[pos] = make_uint2((uint32_t)i, hit);
}

constexpr int kAdjThreads = 128;

// Pass 2 over the touched Gaussians: the sum of their views' adjoints.
__global__ void __launch_bounds__(kAdjThreads, 4) k_adj_multi(
    GeoC geo, const float4* __restrict__ sh, int sh_degree, MultiAdj mv, const uint2* __restrict__ list,
    const int32_t* __restrict__ count, GeoW gw, float4* __restrict__ g_sh) {
  __shared__ float s_sh[48 * kAdjThreads];
  const int cnt = *count;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const uint2 it = list[e];
    const int64_t i = it.x;
    unsigned hit = it.y;
    const float3 mu = geo.mean(i);
    const float3 ls = geo.lsc(i);
    const float4 qr = geo.quat(i);
    const float o = 1.f / (1.f + expf(-geo.opac(i)));
    AdjAcc<SmemSh> acc;
    acc.sh.base = s_sh + threadIdx.x;
    acc.sh.stride = kAdjThreads;
    acc_zero(acc);
    while (hit) {
      const int v = __ffs(hit) - 1;
      hit &= hit - 1;
      const float4* gp = mv.grad2d[v] + 3 * i;
      view_adjoint(mv.cam[v], mu, ls, qr, o, sh + 12 * i, sh_degree, gp[0], gp[1], gp[2],
                   mv.row[v] ? mv.row[v] + 14 * i : nullptr, acc);
    }
    acc_store(acc, i, false, gw, g_sh);
  }
}

// Fused: the adjoint of the touched Gaussians summed over the views, then
// at once the hybrid update of their parameters and moments (modes 0 and 1:
// the update of each Gaussian needs only its own gradient), so the gradient
// never goes to memory.
//
// A block of 128 threads takes 64 list entries a round, in two roles of two
// warps each, so that every Gaussian's adjoint runs as two independent
// chains of about half the length of the whole.  Colour warps (0, 1): the
// colour part of each view's adjoint (SH gradient into a shared-memory
// column, the direction term of the mean's gradient into shared memory),
// the opacity gradient, and the appearance LM block with SH float4 0.
// Geometry warps (2, 3): the geometry part (centre, covariance and
// rotation chain) of the same Gaussians.  After a block barrier the
// geometry warps add the direction term and update the geometry LM block,
// and all four warps run the Adam update of SH float4s 1..11 of the 64
// Gaussians, a quad of lanes on four consecutive float4s of one row (64
// contiguous bytes per Gaussian and load), eight Gaussians per warp, every
// load of a lane issued before its first store.  The column stride
// kShStride = 66 keeps both phases free of shared-memory bank conflicts
// (colour warps: bank 2k + t; Adam phase: bank 8 kk + g8 + const over the
// warp's lanes).  128 registers, four blocks per SM.
constexpr int kUpdG = 64;
constexpr int kShStride = 66;

template <int MODE>
__global__ void __launch_bounds__(kAdjThreads, 4) k_adj_update(
    tgs_param_ptrs P, tgs_param_ptrs M, tgs_param_ptrs V, int64_t n, int sh_degree, MultiAdj mv,
    const uint2* __restrict__ list, const int32_t* __restrict__ count, OptK o) {
  __shared__ float s_sh[48 * kShStride];
  __shared__ float s_dmu[3][kUpdG];
  __shared__ uint32_t s_idx[kUpdG];
  bias_corrections(o);
  const int cnt = *count;
  const GeoC geo = geo_const(geo_of(P));
  const float4* sh = reinterpret_cast<const float4*>(P.sh);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool colour = warp < 2;
  const int t = (warp & 1) * 32 + lane;  // the Gaussian's slot in the round
  const int kk = lane >> 3, g8 = lane & 7;
  for (int b0 = blockIdx.x * kUpdG; b0 < cnt; b0 += gridDim.x * kUpdG) {
    const int e = b0 + t;
    const bool on = e < cnt;
    const uint2 it = on ? list[e] : make_uint2(0u, 0u);
    const int64_t i = it.x;
    unsigned hit = it.y;
    float gg[10];
    if (colour) {
      if (on) {
        s_idx[t] = it.x;
        const float3 mu = geo.mean(i);
        const float o_s = 1.f / (1.f + expf(-geo.opac(i)));
        SmemSh acc_sh{s_sh + t, kShStride};
        acc_sh.zero();
        float og = 0.f, dm[3] = {0.f, 0.f, 0.f};
        while (hit) {
          const int v = __ffs(hit) - 1;
          hit &= hit - 1;
          const float4* gp = mv.grad2d[v] + 3 * i;
          const float4 gb = gp[1], gc = gp[2];
          og += gb.y * o_s * (1.f - o_s);
          float d[3];
          view_colour(mv.cam[v], mu, sh + 12 * i, sh_degree, gb.z, gb.w, gc.x, nullptr, acc_sh, d);
#pragma unroll
          for (int a = 0; a < 3; ++a) dm[a] += d[a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) s_dmu[a][t] = dm[a];
        const float sg[4] = {acc_sh.get(0), acc_sh.get(1), acc_sh.get(2), acc_sh.get(3)};
        lm_update_app<MODE>(P, M, V, n, i, sg, og, nullptr, 0, o);
      }
    } else if (on) {
      const float3 mu = geo.mean(i);
      const float3 ls = geo.lsc(i);
      const float4 qr = geo.quat(i);
#pragma unroll
      for (int a = 0; a < 10; ++a) gg[a] = 0.f;
      while (hit) {
        const int v = __ffs(hit) - 1;
        hit &= hit - 1;
        const float4* gp = mv.grad2d[v] + 3 * i;
        const float4 ga = gp[0];
        const float d_c = gp[1].x;
        float dmu[3], dls[3], dq[4];
        view_geometry(mv.cam[v], mu, ls, qr, ga.x, ga.y, ga.z, ga.w, d_c, dmu, dls, dq);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          gg[a] += dmu[a];
          gg[3 + a] += dls[a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) gg[6 + a] += dq[a];
      }
    }
    __syncthreads();
    if (!colour && on) {
#pragma unroll
      for (int a = 0; a < 3; ++a) gg[a] += s_dmu[a][t];
      lm_update_geo<MODE>(P, M, V, n, i, gg, nullptr, 0, o);
    }
    const int ng = min(kUpdG, cnt - b0);
#pragma unroll 1
    for (int pass = 0; pass < kUpdG / 32; ++pass) {
      const int gl = 32 * pass + 8 * warp + g8;
      if (gl < ng) {
        const int64_t row = 12 * (int64_t)s_idx[gl];
        float4 pp[3], mq[3], vq[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int k4 = kk + 4 * r;
          if (k4 == 0) continue;
          pp[r] = reinterpret_cast<const float4*>(P.sh)[row + k4];
          mq[r] = reinterpret_cast<const float4*>(M.sh)[row + k4];
          vq[r] = reinterpret_cast<const float4*>(V.sh)[row + k4];
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int k4 = kk + 4 * r;
          if (k4 == 0) continue;
          const float* c = s_sh + (4 * k4) * kShStride + gl;
          const float gq[4] = {c[0], c[kShStride], c[2 * kShStride], c[3 * kShStride]};
          float* p4 = &pp[r].x;
          float* m4 = &mq[r].x;
          float* v4 = &vq[r].x;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            moments(gq[u], m4[u], v4[u], o);
            p4[u] += adam_delta(m4[u], v4[u], o.lr[5], o);
          }
          reinterpret_cast<float4*>(P.sh)[row + k4] = pp[r];
          reinterpret_cast<float4*>(M.sh)[row + k4] = mq[r];
          reinterpret_cast<float4*>(V.sh)[row + k4] = vq[r];
        }
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// The fused adjoint + update for geometric fields in 64-byte rows (geo_stride
// 16, rows on 16-byte boundaries).  The same two roles and the same
// arithmetic as k_adj_update, but a round first copies the whole rows it
// needs into shared memory with coalesced asynchronous copies (cp.async):
// the parameters' and both moments' geometric rows, the parameters' SH rows
// and the first view's projected-gradient rows, lanes on consecutive 16-byte
// pieces of a row.  Both roles then read their Gaussian from shared memory,
// the LM steps update the staged geometric rows in place, and the round ends
// by writing those rows back whole, again coalesced.  One thread per
// Gaussian touching its own rows field by field made every warp load and
// store visit 32 scattered rows, and the L1 pipeline that serves them was the
// kernel's limit (71 % busy with DRAM at 31 %).  The unused floats of a row
// (7 and 12..15) are written back with the values read.
constexpr int kRowsG = 64;  // Gaussians a round of the staged-row kernel (128 threads a block)
constexpr int kGeoPad = 20;  // floats per staged geometric row: float4 reads by row are conflict-free
constexpr int kShPad = 52;   // floats per staged SH row

template <int G>
struct __align__(16) AdjRowsSmem {
  float geo[3][G][kGeoPad];  // parameters', first and second moments' geometric rows
  float shp[G][kShPad];      // the parameters' SH rows
  float g2d[G][12];          // the first view's projected-gradient row
  float sh[48 * (G + 2)];    // SH gradient columns (stride G + 2 = 2 mod 8: conflict-free)
  float dmu[3][G];           // direction term of the means' gradient
  uint32_t idx[G];
  uint32_t hit[G];
};

// G Gaussians a round, 2 G threads (G / 32 colour warps, then as many
// geometry warps).
template <int MODE, int G>
__global__ void __launch_bounds__(2 * G, 256 / G) k_adj_update_rows(
    tgs_param_ptrs P, tgs_param_ptrs M, tgs_param_ptrs V, int64_t n, int sh_degree, MultiAdj mv,
    const uint2* __restrict__ list, const int32_t* __restrict__ count, OptK o) {
  constexpr int NT = 2 * G, NW = NT / 32, SS = G + 2;
  __shared__ AdjRowsSmem<G> S;
  bias_corrections(o);
  const int cnt = *count;
  const float4* sh = reinterpret_cast<const float4*>(P.sh);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool colour = warp < NW / 2;
  const int t = (warp % (NW / 2)) * 32 + lane;  // the Gaussian's slot in the round
  const int kk = lane >> 3, g8 = lane & 7;
  for (int b0 = blockIdx.x * G; b0 < cnt; b0 += gridDim.x * G) {
    const int ng = min(G, cnt - b0);
    if (threadIdx.x < G) {
      const uint2 it = threadIdx.x < ng ? list[b0 + threadIdx.x] : make_uint2(0u, 0u);
      S.idx[threadIdx.x] = it.x;
      S.hit[threadIdx.x] = it.y;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < 12 * ng; p += NT) {  // geometric rows: 3 arrays x 4 float4
      const int a = p / (4 * ng), r = p - a * 4 * ng, g = r >> 2, k = r & 3;
      const float* base = a == 0 ? P.means : a == 1 ? M.means : V.means;
      cp_async16(&S.geo[a][g][4 * k], base + 16 * (int64_t)S.idx[g] + 4 * k);
    }
    for (int p = threadIdx.x; p < 12 * ng; p += NT) {  // SH rows: 12 float4
      const int g = p / 12, k = p - 12 * g;
      cp_async16(&S.shp[g][4 * k], sh + 12 * (int64_t)S.idx[g] + k);
    }
    for (int p = threadIdx.x; p < 3 * ng; p += NT) {  // first view's projected gradient: 3 float4
      const int g = p / 3, k = p - 3 * g;
      cp_async16(&S.g2d[g][4 * k], mv.grad2d[__ffs(S.hit[g]) - 1] + 3 * (int64_t)S.idx[g] + k);
    }
    cp_async_commit_wait_all();
    __syncthreads();
    const bool on = t < ng;
    const int64_t i = S.idx[t];
    float gg[10];
    if (colour) {
      if (on) {
        // rows are read and written as float4s (0..3: means, log-scale 0;
        // 4..7: log-scales 1, 2, opacity logit, unused; 8..11: quaternion):
        // scalar accesses at the 20-float row stride would conflict 4 ways
        float4* r1p = reinterpret_cast<float4*>(S.geo[0][t]) + 1;
        float4* r1m = reinterpret_cast<float4*>(S.geo[1][t]) + 1;
        float4* r1v = reinterpret_cast<float4*>(S.geo[2][t]) + 1;
        const float4 r0 = *reinterpret_cast<const float4*>(S.geo[0][t]);
        float4 qp = *r1p, qm = *r1m, qv = *r1v;
        const float3 mu = make_float3(r0.x, r0.y, r0.z);
        const float o_s = 1.f / (1.f + expf(-qp.z));
        SmemSh acc_sh{S.sh + t, SS};
        acc_sh.fresh = true;
        unsigned hit = S.hit[t];
        float og = 0.f, dm[3] = {0.f, 0.f, 0.f};
        while (hit) {
          const int v = __ffs(hit) - 1;
          hit &= hit - 1;
          float4 gb, gc;
          if (acc_sh.fresh) {
            gb = *reinterpret_cast<const float4*>(&S.g2d[t][4]);
            gc = *reinterpret_cast<const float4*>(&S.g2d[t][8]);
          } else {
            const float4* gp = mv.grad2d[v] + 3 * i;
            gb = gp[1];
            gc = gp[2];
          }
          og += gb.y * o_s * (1.f - o_s);
          float d[3];
          view_colour(mv.cam[v], mu, reinterpret_cast<const float4*>(S.shp[t]), sh_degree, gb.z, gb.w, gc.x,
                      nullptr, acc_sh, d);
          acc_sh.fresh = false;
#pragma unroll
          for (int a = 0; a < 3; ++a) dm[a] += d[a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) S.dmu[a][t] = dm[a];
        const float sg[4] = {acc_sh.get(0), acc_sh.get(1), acc_sh.get(2), acc_sh.get(3)};
        const float4 p0 = *reinterpret_cast<const float4*>(S.shp[t]);
        const float4 m0 = reinterpret_cast<const float4*>(M.sh)[12 * i];
        const float4 v0 = reinterpret_cast<const float4*>(V.sh)[12 * i];
        float sp[4] = {p0.x, p0.y, p0.z, p0.w};
        float smm[4] = {m0.x, m0.y, m0.z, m0.w}, sv[4] = {v0.x, v0.y, v0.z, v0.w};
        lm_app_step<MODE>(sg, og, sp, smm, sv, qp.z, qm.z, qv.z, nullptr, 0, n, i, o);
        *r1p = qp;
        *r1m = qm;
        *r1v = qv;
        reinterpret_cast<float4*>(P.sh)[12 * i] = make_float4(sp[0], sp[1], sp[2], sp[3]);
        reinterpret_cast<float4*>(M.sh)[12 * i] = make_float4(smm[0], smm[1], smm[2], smm[3]);
        reinterpret_cast<float4*>(V.sh)[12 * i] = make_float4(sv[0], sv[1], sv[2], sv[3]);
      }
    } else if (on) {
      const float4* pr = reinterpret_cast<const float4*>(S.geo[0][t]);
      const float4 r0 = pr[0], r1 = pr[1], qr = pr[2];
      const float3 mu = make_float3(r0.x, r0.y, r0.z);
      const float3 ls = make_float3(r0.w, r1.x, r1.y);
#pragma unroll
      for (int a = 0; a < 10; ++a) gg[a] = 0.f;
      unsigned hit = S.hit[t];
      bool first = true;
      while (hit) {
        const int v = __ffs(hit) - 1;
        hit &= hit - 1;
        float4 ga;
        float d_c;
        if (first) {
          ga = *reinterpret_cast<const float4*>(&S.g2d[t][0]);
          d_c = S.g2d[t][4];
        } else {
          const float4* gp = mv.grad2d[v] + 3 * i;
          ga = gp[0];
          d_c = gp[1].x;
        }
        first = false;
        float dmu[3], dls[3], dq[4];
        view_geometry(mv.cam[v], mu, ls, qr, ga.x, ga.y, ga.z, ga.w, d_c, dmu, dls, dq);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          gg[a] += dmu[a];
          gg[3 + a] += dls[a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) gg[6 + a] += dq[a];
      }
    }
    __syncthreads();
    if (!colour && on) {
#pragma unroll
      for (int a = 0; a < 3; ++a) gg[a] += S.dmu[a][t];
      float gp[10], gm[10], gv[10];
      float4* rp = reinterpret_cast<float4*>(S.geo[0][t]);
      float4* rm = reinterpret_cast<float4*>(S.geo[1][t]);
      float4* rv = reinterpret_cast<float4*>(S.geo[2][t]);
      auto unpack = [](const float4* r, float (&q)[10]) {
        const float4 a = r[0], b = r[1], c = r[2];
        q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w; q[4] = b.x; q[5] = b.y;
        q[6] = c.x; q[7] = c.y; q[8] = c.z; q[9] = c.w;
      };
      // float 6 (the opacity logit, written by the colour warps) and 7 are re-read and kept
      auto pack = [](const float (&q)[10], float4* r) {
        r[0] = make_float4(q[0], q[1], q[2], q[3]);
        float4 b = r[1];
        b.x = q[4];
        b.y = q[5];
        r[1] = b;
        r[2] = make_float4(q[6], q[7], q[8], q[9]);
      };
      unpack(rp, gp);
      unpack(rm, gm);
      unpack(rv, gv);
      lm_geo_step<MODE>(gg, gp, gm, gv, nullptr, 0, n, i, o);
      pack(gp, rp);
      pack(gm, rm);
      pack(gv, rv);
    }
#pragma unroll 1
    for (int pass = 0; pass < G / (8 * NW); ++pass) {
      const int gl = 8 * NW * pass + 8 * warp + g8;
      if (gl < ng) {
        const int64_t row = 12 * (int64_t)S.idx[gl];
        float4 pp[3], mq[3], vq[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int k4 = kk + 4 * r;
          if (k4 == 0) continue;
          pp[r] = *reinterpret_cast<const float4*>(&S.shp[gl][4 * k4]);
          mq[r] = reinterpret_cast<const float4*>(M.sh)[row + k4];
          vq[r] = reinterpret_cast<const float4*>(V.sh)[row + k4];
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int k4 = kk + 4 * r;
          if (k4 == 0) continue;
          const float* c = S.sh + (4 * k4) * SS + gl;
          const float gq[4] = {c[0], c[SS], c[2 * SS], c[3 * SS]};
          float* p4 = &pp[r].x;
          float* m4 = &mq[r].x;
          float* v4 = &vq[r].x;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            moments(gq[u], m4[u], v4[u], o);
            p4[u] += adam_delta(m4[u], v4[u], o.lr[5], o);
          }
          reinterpret_cast<float4*>(P.sh)[row + k4] = pp[r];
          reinterpret_cast<float4*>(M.sh)[row + k4] = mq[r];
          reinterpret_cast<float4*>(V.sh)[row + k4] = vq[r];
        }
      }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < 12 * ng; p += NT) {  // the updated geometric rows, whole
      const int a = p / (4 * ng), r = p - a * 4 * ng, g = r >> 2, k = r & 3;
      float* base = a == 0 ? P.means : a == 1 ? M.means : V.means;
      *reinterpret_cast<float4*>(base + 16 * (int64_t)S.idx[g] + 4 * k) =
          *reinterpret_cast<const float4*>(&S.geo[a][g][4 * k]);
    }
    __syncthreads();
  }
}

}  // namespace tgs

using namespace tgs;

extern "C" size_t tgs_project_backward_multi_workspace_size(int64_t n) {
  return 256 + sizeof(uint2) * (size_t)std::max<int64_t>(n, 1);
}

extern "C" tgs_status tgs_project_backward_multi(const tgs_gaussians* g, int32_t n_views, const tgs_camera* cams,
                                                 const int32_t* const* radius, const float* const* grad2d,
                                                 const tgs_param_ptrs* grads, uint8_t* touched,
                                                 int32_t write_untouched, float* const* view_rows,
                                                 void* workspace, size_t workspace_bytes, tgs_stream stream) {
  if (!gaussians_ok(g) || n_views < 1 || n_views > kMaxAdjViews || !cams || !radius || !grad2d || !grads)
    return TGS_ERR_INVALID_ARG;
  if (!param_ptrs_ok(grads)) return TGS_ERR_INVALID_ARG;
  if (!workspace || !aligned16(workspace) || workspace_bytes < tgs_project_backward_multi_workspace_size(g->n))
    return TGS_ERR_INVALID_ARG;
  MultiAdj mv;
  mv.n_views = n_views;
  for (int v = 0; v < n_views; ++v) {
    if (!camera_ok(cams + v) || !radius[v] || !grad2d[v] || !aligned16(grad2d[v])) return TGS_ERR_INVALID_ARG;
    float* rw = view_rows ? view_rows[v] : nullptr;
    if (rw && !aligned8(rw)) return TGS_ERR_INVALID_ARG;
    mv.cam[v] = make_cam(cams[v]);
    mv.radius[v] = radius[v];
    mv.grad2d[v] = reinterpret_cast<const float4*>(grad2d[v]);
    mv.row[v] = rw;
  }
  if (g->n == 0) return TGS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* count = reinterpret_cast<int32_t*>(workspace);
  uint2* list = reinterpret_cast<uint2*>(reinterpret_cast<char*>(workspace) + 256);
  cudaMemsetAsync(count, 0, sizeof(int32_t), s);
  k_adj_mark<<<(int)((g->n + 255) / 256), 256, 0, s>>>(g->n, mv, touched, write_untouched, geo_of(*grads),
                                                       reinterpret_cast<float4*>(grads->sh), list, count);
  static int grid_dev[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return TGS_ERR_DEVICE;
  if (!grid_dev[dev]) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_multi, kAdjThreads, 0);
    grid_dev[dev] = std::max(1, sms * std::max(1, per_sm));
  }
  const int grid = (int)std::min<int64_t>(grid_dev[dev], (g->n + kAdjThreads - 1) / kAdjThreads);
  k_adj_multi<<<grid, kAdjThreads, 0, s>>>(geo_of(*g), reinterpret_cast<const float4*>(g->sh), g->sh_degree, mv,
                                           list, count, geo_of(*grads), reinterpret_cast<float4*>(grads->sh));
  return check_launch();
}

extern "C" tgs_status tgs_project_backward_update(const tgs_param_ptrs* params, int64_t n, int32_t sh_degree,
                                                  int32_t n_views, const tgs_camera* cams,
                                                  const int32_t* const* radius, const float* const* grad2d,
                                                  const tgs_param_ptrs* m, const tgs_param_ptrs* v,
                                                  uint8_t* touched, const tgs_opt* opt, int32_t step,
                                                  const int32_t* step_dev, void* workspace, size_t workspace_bytes,
                                                  tgs_stream stream) {
  if (!params || n < 0 || n >= INT32_MAX || sh_degree < 0 || sh_degree > 3 || n_views < 1 ||
      n_views > kMaxAdjViews || !cams || !radius || !grad2d || !m || !v || !opt || step < 1 || opt->mode < 0 ||
      opt->mode > 1 || !(opt->beta1 >= 0.f && opt->beta1 < 1.f) || !(opt->beta2 >= 0.f && opt->beta2 < 1.f))
    return TGS_ERR_INVALID_ARG;
  const tgs_gaussians gs{params->means, params->log_scales, params->quats, params->opacity_logits, params->sh, n,
                         sh_degree, params->geo_stride};
  const tgs_gaussians* g = &gs;
  if (!gaussians_ok(g)) return TGS_ERR_INVALID_ARG;
  for (const tgs_param_ptrs* q : {m, v})
    if (!param_ptrs_ok(q)) return TGS_ERR_INVALID_ARG;
  if (!workspace || !aligned16(workspace) || workspace_bytes < tgs_project_backward_multi_workspace_size(g->n))
    return TGS_ERR_INVALID_ARG;
  MultiAdj mv;
  mv.n_views = n_views;
  for (int k = 0; k < n_views; ++k) {
    if (!camera_ok(cams + k) || !radius[k] || !grad2d[k] || !aligned16(grad2d[k])) return TGS_ERR_INVALID_ARG;
    mv.cam[k] = make_cam(cams[k]);
    mv.radius[k] = radius[k];
    mv.grad2d[k] = reinterpret_cast<const float4*>(grad2d[k]);
    mv.row[k] = nullptr;
  }
  if (g->n == 0) return TGS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* count = reinterpret_cast<int32_t*>(workspace);
  uint2* list = reinterpret_cast<uint2*>(reinterpret_cast<char*>(workspace) + 256);
  cudaMemsetAsync(count, 0, sizeof(int32_t), s);
  // the mark pass writes no gradients (nothing to zero)
  k_adj_mark<<<(int)((g->n + 255) / 256), 256, 0, s>>>(g->n, mv, touched, 0, GeoW{}, nullptr, list, count);
  // 64-byte geometric rows on 16-byte boundaries in all three: the staged-row kernel
  const bool rows = params->geo_stride == 16 && m->geo_stride == 16 && v->geo_stride == 16 &&
                    aligned16(params->means) && aligned16(m->means) && aligned16(v->means);
  static int grid_dev[64][2][2] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return TGS_ERR_DEVICE;
  const int md = opt->mode;
  int& gd = grid_dev[dev][md][rows ? 1 : 0];
  if (!gd) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* fn = rows ? (md == 0 ? (const void*)k_adj_update_rows<0, kRowsG> : (const void*)k_adj_update_rows<1, kRowsG>)
                          : (md == 0 ? (const void*)k_adj_update<0> : (const void*)k_adj_update<1>);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, rows ? 2 * kRowsG : kAdjThreads, 0);
    gd = std::max(1, sms * std::max(1, per_sm));
  }
  const int per_round = rows ? kRowsG : kUpdG;
  const int grid = (int)std::min<int64_t>(gd, (g->n + per_round - 1) / per_round);
  const tgs_param_ptrs P = *params;
  const OptK o = make_optk(opt, step, step_dev);
  if (rows) {
    if (md == 0)
      k_adj_update_rows<0, kRowsG><<<grid, 2 * kRowsG, 0, s>>>(P, *m, *v, g->n, g->sh_degree, mv, list, count, o);
    else
      k_adj_update_rows<1, kRowsG><<<grid, 2 * kRowsG, 0, s>>>(P, *m, *v, g->n, g->sh_degree, mv, list, count, o);
  } else if (md == 0) {
    k_adj_update<0><<<grid, kAdjThreads, 0, s>>>(P, *m, *v, g->n, g->sh_degree, mv, list, count, o);
  } else {
    k_adj_update<1><<<grid, kAdjThreads, 0, s>>>(P, *m, *v, g->n, g->sh_degree, mv, list, count, o);
  }
  return check_launch();
}

namespace tgs {

bool gaussians_ok(const tgs_gaussians* g) {
  if (!g || g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3 || !geo_stride_ok(g->geo_stride)) return false;
  if (g->n == 0) return true;
  return g->means && g->log_scales && g->quats && g->opacity_logits && g->sh && aligned4(g->means) &&
         aligned4(g->log_scales) && aligned16(g->quats) && aligned4(g->opacity_logits) && aligned16(g->sh);
}

bool camera_ok(const tgs_camera* c) {
  return c && c->width > 0 && c->height > 0 && c->fx > 0.f && c->fy > 0.f && c->znear > 0.f &&
         c->width <= (1 << 16) && c->height <= (1 << 16);
}

}  // namespace tgs

using namespace tgs;

extern "C" tgs_status tgs_project_gaussians(const tgs_gaussians* g, const tgs_camera* cam, const int32_t* tile_rank,
                                            tgs_projected* out, tgs_stream stream) {
  if (!gaussians_ok(g) || !camera_ok(cam) || !out) return TGS_ERR_INVALID_ARG;
  if (g->n == 0) return TGS_OK;
  if (!out->xy || !out->conic_opac || !out->rgb || !out->depth || !out->radius || !aligned8(out->xy) ||
      !aligned16(out->conic_opac))
    return TGS_ERR_INVALID_ARG;
  CamK k = make_cam(*cam);
  int blocks = (int)((g->n + 255) / 256);
  k_project<<<blocks, 256, 0, (cudaStream_t)stream>>>(
      geo_of(*g), reinterpret_cast<const float4*>(g->sh), g->n, g->sh_degree, k, tile_rank,
      reinterpret_cast<float2*>(out->xy), reinterpret_cast<float4*>(out->conic_opac), out->rgb, out->depth,
      out->radius);
  return check_launch();
}
