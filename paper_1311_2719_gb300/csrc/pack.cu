// Link preparation (the paper's linkc_acc, §4) and canonical <-> packed field conversion.
#include "dslash.cuh"

namespace qcd {

// One thread per (parity, mu, even-odd site). Reads the canonical link U_mu(n) of site n and
// stores it in the packed layout of (PREC, RECON).
template <int PREC, int RECON>
__global__ void pack_links_kernel(Geom g, const double2* __restrict__ canon, void* __restrict__ out) {
  const long long total = 8ll * g.Vh;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t % g.Vh);
    const int pm = (int)(t / g.Vh);  // par * 4 + mu
    const int par = pm >> 2, mu = pm & 3;
    const Site s = site_of(g, k, par);
    const double2* src = canon + ((size_t)s.lex * 4 + mu) * 9;
    double2 e[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) e[i] = src[i];
    if constexpr (RECON == 18) {
      const double f = 0.5 * (double)fwd_sign(g, s, mu);
#pragma unroll
      for (int i = 0; i < 9; ++i) e[i] = make_double2(f * e[i].x, f * e[i].y);
      if constexpr (PREC == QCD_PREC_DOUBLE) {
        double2* o = (double2*)out + (size_t)pm * 9 * g.Vh + k;
#pragma unroll
        for (int i = 0; i < 9; ++i) o[(size_t)i * g.Vh] = e[i];
      } else if constexpr (PREC == QCD_PREC_DF64) {
        float4* o = (float4*)out + (size_t)pm * 9 * g.Vh + k;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const df64 re(e[i].x), im(e[i].y);
          o[(size_t)i * g.Vh] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
      } else {
        float2* o = (float2*)out + (size_t)pm * 9 * g.Vh + k;
#pragma unroll
        for (int i = 0; i < 9; ++i) o[(size_t)i * g.Vh] = make_float2((float)e[i].x, (float)e[i].y);
      }
    } else {  // RECON == 12: rows 0 and 1, unphased
      if constexpr (PREC == QCD_PREC_SINGLE) {
        float4* o = (float4*)out + (size_t)pm * 3 * g.Vh + k;
        o[0] = make_float4((float)e[0].x, (float)e[0].y, (float)e[1].x, (float)e[1].y);
        o[(size_t)g.Vh] = make_float4((float)e[2].x, (float)e[2].y, (float)e[3].x, (float)e[3].y);
        o[2 * (size_t)g.Vh] = make_float4((float)e[4].x, (float)e[4].y, (float)e[5].x, (float)e[5].y);
      } else {
        uint4* oa = (uint4*)out + (size_t)pm * g.Vh + k;
        uint2* ob = (uint2*)((uint4*)out + 8 * (size_t)g.Vh) + (size_t)pm * g.Vh + k;
        unsigned w[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) w[i] = float2_to_fx16x2((float)e[i].x, (float)e[i].y);
        *oa = make_uint4(w[0], w[1], w[2], w[3]);
        *ob = make_uint2(w[4], w[5]);
      }
    }
  }
}

int launch_pack_links(const qcd_lattice* lat, const void* canon, void* out, int prec, int recon, cudaStream_t st) {
  const Geom g = make_geom(lat);
  const long long total = 8ll * g.Vh;
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 64) grid = 152 * 64;
  const double2* c = (const double2*)canon;
  if (prec == QCD_PREC_DOUBLE && recon == 18) pack_links_kernel<QCD_PREC_DOUBLE, 18><<<grid, 256, 0, st>>>(g, c, out);
  else if (prec == QCD_PREC_SINGLE && recon == 18) pack_links_kernel<QCD_PREC_SINGLE, 18><<<grid, 256, 0, st>>>(g, c, out);
  else if (prec == QCD_PREC_SINGLE && recon == 12) pack_links_kernel<QCD_PREC_SINGLE, 12><<<grid, 256, 0, st>>>(g, c, out);
  else if (prec == QCD_PREC_HALF && recon == 12) pack_links_kernel<QCD_PREC_HALF, 12><<<grid, 256, 0, st>>>(g, c, out);
  else if (prec == QCD_PREC_DF64 && recon == 18) pack_links_kernel<QCD_PREC_DF64, 18><<<grid, 256, 0, st>>>(g, c, out);
  else return QCD_ERR_UNSUPPORTED;
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

// canonical complex128[V][3] <-> packed field of one parity. One thread per even-odd site.
template <int PREC>
__global__ void pack_field_kernel(Geom g, Field<PREC> out, const double2* __restrict__ canon, int par) {
  using T = typename Field<PREC>::T;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.Vh; k += gridDim.x * blockDim.x) {
    const Site s = site_of(g, k, par);
    cvec3<T> v;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double2 d = canon[(size_t)s.lex * 3 + a];
      v.c[a].re = (T)d.x; v.c[a].im = (T)d.y;
    }
    out.store(k, v);
  }
}

template <int PREC>
__global__ void unpack_field_kernel(Geom g, double2* __restrict__ canon, Field<PREC> in, int par) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.Vh; k += gridDim.x * blockDim.x) {
    const Site s = site_of(g, k, par);
    auto v = in.load(k);
#pragma unroll
    for (int a = 0; a < 3; ++a) canon[(size_t)s.lex * 3 + a] = make_double2((double)v.c[a].re, (double)v.c[a].im);
  }
}

int launch_pack_field(const qcd_lattice* lat, void* packed, const void* canon, int par, int prec, cudaStream_t st) {
  const Geom g = make_geom(lat);
  const int grid = site_grid(g.Vh);
  const double2* c = (const double2*)canon;
  switch (prec) {
    case QCD_PREC_DOUBLE: pack_field_kernel<<<grid, kBlock, 0, st>>>(g, make_field<QCD_PREC_DOUBLE>(packed, g.Vh), c, par); break;
    case QCD_PREC_SINGLE: pack_field_kernel<<<grid, kBlock, 0, st>>>(g, make_field<QCD_PREC_SINGLE>(packed, g.Vh), c, par); break;
    case QCD_PREC_HALF: pack_field_kernel<<<grid, kBlock, 0, st>>>(g, make_field<QCD_PREC_HALF>(packed, g.Vh), c, par); break;
    case QCD_PREC_DF64: pack_field_kernel<<<grid, kBlock, 0, st>>>(g, make_field<QCD_PREC_DF64>(packed, g.Vh), c, par); break;
    default: return QCD_ERR_INVALID_ARG;
  }
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

int launch_unpack_field(const qcd_lattice* lat, void* canon, const void* packed, int par, int prec, cudaStream_t st) {
  const Geom g = make_geom(lat);
  const int grid = site_grid(g.Vh);
  double2* c = (double2*)canon;
  void* p = const_cast<void*>(packed);
  switch (prec) {
    case QCD_PREC_DOUBLE: unpack_field_kernel<<<grid, kBlock, 0, st>>>(g, c, make_field<QCD_PREC_DOUBLE>(p, g.Vh), par); break;
    case QCD_PREC_SINGLE: unpack_field_kernel<<<grid, kBlock, 0, st>>>(g, c, make_field<QCD_PREC_SINGLE>(p, g.Vh), par); break;
    case QCD_PREC_HALF: unpack_field_kernel<<<grid, kBlock, 0, st>>>(g, c, make_field<QCD_PREC_HALF>(p, g.Vh), par); break;
    case QCD_PREC_DF64: unpack_field_kernel<<<grid, kBlock, 0, st>>>(g, c, make_field<QCD_PREC_DF64>(p, g.Vh), par); break;
    default: return QCD_ERR_INVALID_ARG;
  }
  QCD_CUDA(cudaGetLastError());
  return QCD_OK;
}

}  // namespace qcd
