// fdlb_kernels.cu -- sm_103a kernels of the IMEX finite-difference lattice
// Boltzmann step (Kis & Ambrus): one fused kernel per advected IMEX stage.
//
// Every stage kernel owns a tile of cells and all populations of those cells,
// and runs two passes:
//   pass 1  for each group of G populations: stage the advected array on the
//           tile plus its 5-cell MP-9 halo in shared memory (ghosts by index
//           clamp = outlet copies of the adjacent fluid node, Sec. IV), march
//           every tile line computing each interface value once (MP-9 + MP
//           limiter, fdlb_mp9.cuh), form the flux difference and the explicit
//           part R_i of the stage (Eq. IMEX), accumulate the moments of R_i
//           per cell (Eq. Moments_discrete) and park R_i and the running
//           accumulators in the output arrays;
//   pass 2  per cell: n, u, T from the moments, the Hermite equilibrium
//           factors (Eq. gExpanded, recurrence form), and the closed-form
//           implicit BGK relaxation of every population (Sec. III).  Stages
//           3 and 4 leave D_i = R_i - F_eq(R_i) in the array D, which the
//           next kernel folds into A4 and A_fin in its pass 1, so that pass 2
//           rewrites the relaxed populations and D only.
// The flux itself never goes to global memory.
#include "fdlb_device.cuh"

namespace fdlb {
namespace {

// One tile (origin x0, y0 of problem g) of one fused stage; see the file
// header for the two passes.  Ends with every thread past its last use of
// the shared memory, so a persistent CTA may start its next tile at once.
template <int DIM, int QP, int QC, int STAGE, typename S, int VAR>
__device__ __forceinline__ void stage_tile(const DevParams& p, const Geo& geo, int x0, int y0,
                                           TileSmem<DIM, S, VAR>& sm) {
  using C = TileCfg<DIM, VAR>;
  using L = Lat<DIM, QP, QC>;
  constexpr int TX = C::TX, TY = C::TY, NT = C::NT, G = C::G, SEG = C::SEG;
  constexpr int SX = TileSmem<DIM, S, VAR>::SX;
  constexpr int CELLS = TX * TY;
  constexpr int CPT = (CELLS + NT - 1) / NT;
  constexpr int NSEG = (TX + 1) / SEG;  // segments per line
  static_assert(NSEG * SEG == TX + 1, "segments tile the line");
  constexpr int NLINE = DIM == 2 ? TX + TY : 1;
  static_assert(G * NLINE * NSEG == NT, "one march task per thread");

  constexpr int SY = TileSmem<DIM, S, VAR>::SY;
  auto& tile = sm.tile;
  auto& hx = sm.hx;
  auto& hy = sm.hy;
  S* __restrict__ const F = (S*)p.F;
  S* __restrict__ const F2 = (S*)p.F2;
  S* __restrict__ const F3 = (S*)p.F3;
  S* __restrict__ const A4 = (S*)p.A4;
  S* __restrict__ const Af = (S*)p.Af;
  S* __restrict__ const Dn = (S*)p.D;

  const int tid = threadIdx.x;
  const int64_t N = p.N;  // population stride

  int lxs[CPT], lys[CPT];
  int64_t cell[CPT];
  bool valid[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int c = tid + k * NT;
    lxs[k] = c % TX;
    lys[k] = c / TX;
    const int x = x0 + lxs[k], y = y0 + lys[k];
    valid[k] = (c < CELLS) && (x < geo.nx) && (y < geo.ny);
    cell[k] = geo.base + (int64_t)y * geo.nx + x;
  }
  typename MomAcc<S>::type mom[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) mom[k] = {};

  const CoefS<S> sc(p.sc);

  if (STAGE == kPrep) {
    for (int pop = 0; pop < L::P; ++pop) {
#pragma unroll
      for (int k = 0; k < CPT; ++k)
        if (valid[k]) accumulate<DIM, QP, QC>(p, mom[k], pop, F[pop * N + cell[k]]);
    }
  } else {
    const S* __restrict__ adv = (STAGE == kStage3) ? F2 : (STAGE == kStage4) ? F3 : A4;
    // this thread's march task: population tg of the group, line, segment
    const int tg = tid / (NLINE * NSEG);
    const int tline = (tid / NSEG) % NLINE;
    // this thread's staged cells (tile offset, cell offset from geo.base or
    // -1): ghosts by index clamp or wrap; the 2-D halo corners feed no line
    constexpr int SXH = TX + 2 * H;
    constexpr int NST = SY * SXH;
    constexpr int J = (NST + NT - 1) / NT;
    int soff[J], goff[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int e = tid + j * NT;
      const int r = e / SXH, c = e % SXH;
      soff[j] = r * SX + c;
      goff[j] = -1;
      const bool corner = DIM == 2 && (r < H || r >= H + TY) && (c < H || c >= H + TX);
      if (e < NST && !corner) {
        const int gx = wrap_or_clamp(x0 - H + c, geo.nx, p.bc);
        const int gy = (DIM == 2) ? wrap_or_clamp(y0 - H + r, geo.ny, p.bc) : 0;
        goff[j] = gy * geo.nx + gx;
      }
    }
    // the group's advected populations on tile + halo, copied asynchronously;
    // the next group's copies run during this group's pass 1
    auto prefetch = [&](int gfirst) {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int pop = gfirst + g;
        if (pop >= L::P) break;
        const S* __restrict__ src = adv + (int64_t)pop * N + geo.base;
#pragma unroll
        for (int j = 0; j < J; ++j)
          if (goff[j] >= 0) cp_async(&tile[g][0][0] + soff[j], src + goff[j]);
      }
      cp_async_commit();
    };
    prefetch(0);
    for (int g0 = 0; g0 < L::P; g0 += G) {
      cp_async_wait_all();
      __syncthreads();  // the group's tile is in; the previous pass 1 is done
      // ---- every interface value once, marching upwind -> downwind
      {
        const int pop = g0 + tg;
        const bool xline = (DIM == 1) || (tline < TY);
        const double pv = (pop < L::P) ? (xline ? p.px[pop] : p.py[pop]) : 0.0;
        const int sgn = (pv >= 0.0) ? 1 : -1;
        // one call site for x and y lines (a warp holds both kinds): the line
        // is (base, signed element stride) in the tile and its output slots
        // (march_task: interface i lies between tile cells i-1 and i, tile
        // cell c at column/row c + H, mirror image for p < 0)
        const MarchTask t = march_task(tid, DIM, TX, TY, SEG, SX, sgn);
        S* out = t.xline ? &hx[tg][t.orow][t.ofirst] : &hy[tg][t.orow][t.ofirst];
        mp9_march<SEG>(&tile[tg][t.br][t.bc_], t.stride, out, sgn);
      }
      __syncthreads();  // the march is done with the tile
      if (g0 + G < L::P) prefetch(g0 + G);
      // ---- flux difference, explicit part, moments (pass 1)
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        if (!valid[k]) continue;
        const int lx = lxs[k], ly = lys[k];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int pop = g0 + g;
          if (pop >= L::P) break;
          // X = dt * (p . grad F) = dt p_x (Fhat_{x+1/2} - Fhat_{x-1/2})/dx + (y);
          // single problems use the host's dt p/dx (the same product)
          const double cxv = geo.prob < 0 ? p.cx[pop] : geo.dtdx * p.px[pop];
          S X = (S)cxv * (hx[g][ly][lx + 1] - hx[g][ly][lx]);
          if constexpr (DIM == 2) {
            const double cyv = geo.prob < 0 ? p.cy[pop] : geo.dtdy * p.py[pop];
            X = sfma((S)cyv, hy[g][lx][ly + 1] - hy[g][lx][ly], X);
          }
          const int64_t e = pop * N + cell[k];
          S R;
          if (STAGE == kStage3) {
            const S f = F[e], dd = Dn[e];
            R = sfma(-sc.at32, X, sfma(-sc.k3, dd, f));
            F3[e] = R;
            A4[e] = sfma(-sc.at42, X, sfma(-sc.k4, dd, f));
            Af[e] = sfma(-sc.wt2, X, sfma(-sc.kf, dd, f));
          } else if (STAGE == kStage4) {
            // the D3 terms of A4 and A_fin, left by stage 3 in D
            const S d3 = Dn[e];
            R = sfma(-sc.at43, X, sfma(-sc.a43e3, d3, A4[e]));
            A4[e] = R;
            Af[e] = sfma(-sc.wt3, X, sfma(-sc.w3e3, d3, Af[e]));
          } else {  // kFinal: F^{n+1}, with the D4 term left by stage 4 in D
            R = sfma(-sc.wt4, X, sfma(-sc.w4e4, Dn[e], Af[e]));
            F[e] = R;
          }
          accumulate<DIM, QP, QC>(p, mom[k], pop, R);
        }
      }
    }
    __syncthreads();  // every thread past its last use of hx, hy
  }

  // ---- pass 2: equilibrium of the moments and closed-form relaxation
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    if (!valid[k]) continue;
    double n, ux, uy, T;
    if (!moments_to_nut<DIM>(geo.invDK, to_fp64(mom[k]), n, ux, uy, T)) {
      atomicOr(p.status, 1u);
      if (geo.prob >= 0) atomicOr(&p.pstatus[geo.prob], 1u);
    }
    EqCell<DIM, QP, QC> eq64;
    make_eq_nut<DIM, QP, QC>(p, geo.kchi, n, ux, uy, T, eq64);
    EqCellS<DIM, QP, QC, S> eq;
    to_storage(eq64, eq);
    const int64_t c = cell[k];
#pragma unroll
    for (int pop = 0; pop < L::P; ++pop) {
      const int64_t e = pop * N + c;
      const S fe = feq_of<DIM, QP, QC, S>(eq, pop);
      if (STAGE == kStage3) {
        // F3 relaxed; D3 goes to D (free until the final stage rewrites it),
        // and stage 4 applies its terms to A4 and A_fin as it reads them
        const S R = F3[e];
        const S D3 = R - fe;
        F3[e] = sfma(-sc.a33e3, D3, R);
        Dn[e] = D3;
      } else if (STAGE == kStage4) {
        // F4 relaxed; D4 goes to D for the final stage's A_fin
        const S R = A4[e];
        const S D4 = R - fe;
        A4[e] = sfma(-sc.a44e4, D4, R);
        Dn[e] = D4;
      } else {  // kPrep / kFinal: D and F2 of the new state
        const S f = F[e];
        const S dd = f - fe;
        Dn[e] = dd;
        F2[e] = sfma(sc.c2, dd, fe);
      }
    }
  }
}

// One tile per CTA, the grid covering one problem.
template <int DIM, int QP, int QC, int STAGE, typename S, int VAR = 0>
__global__ void __launch_bounds__(TileCfg<DIM, VAR>::NT)
    stage_kernel(const __grid_constant__ DevParams p) {
  __shared__ TileSmem<DIM, S, VAR> sm;
  const Geo geo{p.nx, p.ny, 0, p.kchi, p.invDK, p.dtdx, p.dtdy, -1};
  stage_tile<DIM, QP, QC, STAGE, S, VAR>(p, geo, blockIdx.x * TileCfg<DIM, VAR>::TX,
                                         blockIdx.y * TileCfg<DIM, VAR>::TY, sm);
}

// Batches of 1-D problems: a persistent grid walks the tile work list of all
// problems (each tile within one problem, ghosts clamped at its own ends).
template <int QP, int QC, int STAGE, typename S, int VAR>
__global__ void __launch_bounds__(TileCfg<1, VAR>::NT)
    batch_stage_kernel(const __grid_constant__ DevParams p) {
  __shared__ TileSmem<1, S, VAR> sm;
  for (int w = blockIdx.x; w < p.nwork; w += gridDim.x) {
    const WorkItem it = p.work[w];
    const BatchProblem& bp = p.probs[it.prob];
    const Geo geo{bp.nx, 1, bp.base, bp.kchi, bp.invDK, bp.dtdx, 0.0, it.prob};
    stage_tile<1, QP, QC, STAGE, S, VAR>(p, geo, it.x0, 0, sm);
  }
}

// Store the binary64 equilibrium of cell c as the state: binary64 values
// (FDLB_FP64), or binary32 pairs hi + lo with hi the rounded value and lo
// the rounded remainder (FDLB_MIXED).
template <typename S, int DIM, int QP, int QC>
__device__ __forceinline__ void store_state(const DevParams& p,
                                            const EqCellS<DIM, QP, QC, double>& eq, int64_t c) {
  using L = Lat<DIM, QP, QC>;
#pragma unroll
  for (int pop = 0; pop < L::P; ++pop) {
    const double v = feq_of<DIM, QP, QC, double>(eq, pop);
    if constexpr (sizeof(S) == 8) {
      ((double*)p.F)[pop * p.N + c] = v;
    } else {
      const float h = (float)v;
      p.sh[pop * p.N + c] = h;
      p.sl[pop * p.N + c] = (float)(v - (double)h);
    }
  }
}

// problem of cell c (problems sorted by base)
__device__ __forceinline__ int find_problem(const DevParams& p, int64_t c) {
  int lo = 0, hi = p.nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (p.probs[mid].base <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int QP, int QC, typename S>
__global__ void batch_init_kernel(const __grid_constant__ DevParams p) {
  using L = Lat<1, QP, QC>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const BatchProblem& bp = p.probs[find_problem(p, c)];
  const int x = (int)(c - bp.base);
  const int q = ((double)x + 0.5 >= bp.split) ? 1 : 0;
  const double rho = bp.st[q][0], ux = bp.st[q][1], P = bp.st[q][2];
  EqCell<1, QP, QC> eq64;
  make_eq_nut<1, QP, QC>(p, bp.kchi, rho, ux, 0.0, P / rho, eq64);
  EqCellS<1, QP, QC, double> eq;
  to_storage(eq64, eq);
  store_state<S>(p, eq, c);
}

// Piecewise-constant Riemann data -> discrete equilibrium (Sec. V).
struct RiemannArgs {
  double st[4][4];
  int nq;
  double sx, sy;  // membranes in cell units (split_in_cells)
};

template <int DIM, int QP, int QC, typename S>
__global__ void init_riemann_kernel(const __grid_constant__ DevParams p,
                                    const __grid_constant__ RiemannArgs a) {
  using L = Lat<DIM, QP, QC>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const int x = (int)(c % p.nx), y = (int)(c / p.nx);
  const bool right = (double)x + 0.5 >= a.sx;
  int q;
  if (DIM == 1) {
    q = right ? 1 : 0;
  } else {
    const bool upper = (double)y + 0.5 >= a.sy;
    q = upper ? (right ? 0 : 1) : (right ? 3 : 2);
  }
  const double rho = a.st[q][0];
  const double ux = a.st[q][1];
  const double uy = DIM == 2 ? a.st[q][2] : 0.0;
  const double P = a.st[q][DIM == 2 ? 3 : 2];
  EqCell<DIM, QP, QC> eq64;
  make_eq_nut<DIM, QP, QC>(p, p.kchi, rho, ux, uy, P / rho, eq64);
  EqCellS<DIM, QP, QC, double> eq;  // binary64 products, rounded once on store
  to_storage(eq64, eq);
  store_state<S>(p, eq, c);
}

// Moments of a binary32-pair state: the binary64 sums of the high parts
// (mhi, kept by the stage kernels) plus binary64 sums of the low parts.
template <int DIM, int QP, int QC>
__global__ void mixed_moments_kernel(const __grid_constant__ DevParams p, double* __restrict__ n,
                                     double* __restrict__ ux, double* __restrict__ uy,
                                     double* __restrict__ T) {
  using L = Lat<DIM, QP, QC>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  Moments m = {p.mhi[c], p.mhi[p.N + c], p.mhi[2 * p.N + c], p.mhi[3 * p.N + c]};
  for (int pop = 0; pop < L::P; ++pop) accumulate<DIM, QP, QC>(p, m, pop, (double)p.sl[pop * p.N + c]);
  double nn, vx, vy, TT;
  const double invDK = p.nprob > 0 ? p.probs[find_problem(p, c)].invDK : p.invDK;
  moments_to_nut<DIM>(invDK, m, nn, vx, vy, TT);
  n[c] = nn;
  ux[c] = vx;
  if (DIM == 2 && uy) uy[c] = vy;
  T[c] = TT;
}

template <int DIM, int QP, int QC, typename S>
__global__ void moments_kernel(const __grid_constant__ DevParams p, double* __restrict__ n,
                               double* __restrict__ ux, double* __restrict__ uy,
                               double* __restrict__ T) {
  using L = Lat<DIM, QP, QC>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  typename MomAcc<S>::type m = {};
  const S* F = (const S*)p.F;
  for (int pop = 0; pop < L::P; ++pop) accumulate<DIM, QP, QC>(p, m, pop, F[pop * p.N + c]);
  double nn, vx, vy, TT;
  const double invDK = p.nprob > 0 ? p.probs[find_problem(p, c)].invDK : p.invDK;
  moments_to_nut<DIM>(invDK, to_fp64(m), nn, vx, vy, TT);
  n[c] = nn;
  ux[c] = vx;
  if (DIM == 2 && uy) uy[c] = vy;
  T[c] = TT;
}

// Transpose of the moment map (n, u, T)(F) of Eq. (Moments_discrete) at the
// current binary64 state: with n = sum phi, u = j/n, j = sum phi p and
// T = (e - n u^2)/((D+K) n), e = sum phi p^2 + sum chi,
//   dn/dphi_k = 1,  du_a/dphi_k = (p_a,k - u_a)/n,
//   dT/dphi_k = (|p_k - u|^2 - (D+K) T)/((D+K) n),  dT/dchi_q = 1/((D+K) n),
// so Fbar = J^T (nbar, ubar, Tbar) (absent adjoints are zero).  The state is
// read only when ubar or Tbar is given: n is linear in F.
template <int DIM, int QP, int QC>
__global__ void moments_adjoint_kernel(const __grid_constant__ DevParams p,
                                       const double* __restrict__ nbar,
                                       const double* __restrict__ uxbar,
                                       const double* __restrict__ uybar,
                                       const double* __restrict__ Tbar, double* __restrict__ Fbar) {
  using L = Lat<DIM, QP, QC>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const double nb = nbar ? nbar[c] : 0.0;
  const double uxb = uxbar ? uxbar[c] : 0.0;
  const double uyb = (DIM == 2 && uybar) ? uybar[c] : 0.0;
  const double Tb = Tbar ? Tbar[c] : 0.0;
  double nn = 1.0, vx = 0.0, vy = 0.0, TT = 0.0;
  if (uxbar || (DIM == 2 && uybar) || Tbar) {
    Moments m = {};
    const double* F = (const double*)p.F;
    for (int pop = 0; pop < L::P; ++pop) accumulate<DIM, QP, QC>(p, m, pop, F[pop * p.N + c]);
    moments_to_nut<DIM>(p.invDK, m, nn, vx, vy, TT);
  }
  const double inv_n = 1.0 / nn;
  const double tq = Tb * p.invDK * inv_n;  // Tbar / ((D+K) n)
  for (int pop = 0; pop < L::P; ++pop) {
    double v;
    if (pop < L::NPHI) {
      const double dx = p.px[pop] - vx, dy = DIM == 2 ? p.py[pop] - vy : 0.0;
      v = nb + (uxb * dx + uyb * dy) * inv_n + tq * (dx * dx + dy * dy - p.DK * TT);
    } else {
      v = tq;
    }
    Fbar[pop * p.N + c] = v;
  }
}

template <int DIM, int QP, int QC, typename S, int VAR>
int launch_stage_tsv(const DevParams& p, int stage, cudaStream_t s) {
  using C = TileCfg<DIM, VAR>;
  dim3 grid((p.nx + C::TX - 1) / C::TX, DIM == 2 ? (p.ny + C::TY - 1) / C::TY : 1);
  switch (stage) {
    case kPrep: stage_kernel<DIM, QP, QC, kPrep, S, VAR><<<grid, C::NT, 0, s>>>(p); break;
    case kStage3: stage_kernel<DIM, QP, QC, kStage3, S, VAR><<<grid, C::NT, 0, s>>>(p); break;
    case kStage4: stage_kernel<DIM, QP, QC, kStage4, S, VAR><<<grid, C::NT, 0, s>>>(p); break;
    default: stage_kernel<DIM, QP, QC, kFinal, S, VAR><<<grid, C::NT, 0, s>>>(p); break;
  }
  return (int)cudaGetLastError();
}

// 1-D problems pick their tile shape by length (single_1d_variant).
template <int DIM, int QP, int QC, typename S>
int launch_stage_ts(const DevParams& p, int stage, cudaStream_t s) {
  if constexpr (DIM == 1) {
    switch (single_1d_variant(p.nx)) {
      case 1: return launch_stage_tsv<1, QP, QC, S, 1>(p, stage, s);
      case 3: return launch_stage_tsv<1, QP, QC, S, 3>(p, stage, s);
      case 4: return launch_stage_tsv<1, QP, QC, S, 4>(p, stage, s);
      default: return launch_stage_tsv<1, QP, QC, S, 0>(p, stage, s);
    }
  }
  return launch_stage_tsv<DIM, QP, QC, S, 0>(p, stage, s);
}

template <int DIM, int QP, int QC>
int launch_stage_t(const DevParams& p, int stage, cudaStream_t s) {
  // binary32 contexts run the single-pass kernels of fdlb_mixed.cu
  return p.precision == 1 ? launch_mixed_stage(p, stage, s)
                          : launch_stage_ts<DIM, QP, QC, double>(p, stage, s);
}

template <int DIM, int QP, int QC>
int launch_init_t(const DevParams& p, const RiemannArgs& a, cudaStream_t s) {
  const int nt = 128;
  const int64_t nb = (p.N + nt - 1) / nt;
  if (p.precision == 1) init_riemann_kernel<DIM, QP, QC, float><<<(unsigned)nb, nt, 0, s>>>(p, a);
  else init_riemann_kernel<DIM, QP, QC, double><<<(unsigned)nb, nt, 0, s>>>(p, a);
  return (int)cudaGetLastError();
}

template <int DIM, int QP, int QC>
int launch_moments_t(const DevParams& p, double* n, double* ux, double* uy, double* T,
                     cudaStream_t s) {
  const int nt = 128;
  const int64_t nb = (p.N + nt - 1) / nt;
  if (p.precision == 1) mixed_moments_kernel<DIM, QP, QC><<<(unsigned)nb, nt, 0, s>>>(p, n, ux, uy, T);
  else moments_kernel<DIM, QP, QC, double><<<(unsigned)nb, nt, 0, s>>>(p, n, ux, uy, T);
  return (int)cudaGetLastError();
}

template <int QP, int QC, typename S, int VAR>
int launch_batch_stage_v(const DevParams& p, int stage, cudaStream_t s) {
  using C = TileCfg<1, VAR>;
  const int grid = p.bgrid > 0 ? p.bgrid : 1;
  switch (stage) {
    case kPrep: batch_stage_kernel<QP, QC, kPrep, S, VAR><<<grid, C::NT, 0, s>>>(p); break;
    case kStage3: batch_stage_kernel<QP, QC, kStage3, S, VAR><<<grid, C::NT, 0, s>>>(p); break;
    case kStage4: batch_stage_kernel<QP, QC, kStage4, S, VAR><<<grid, C::NT, 0, s>>>(p); break;
    default: batch_stage_kernel<QP, QC, kFinal, S, VAR><<<grid, C::NT, 0, s>>>(p); break;
  }
  return (int)cudaGetLastError();
}

template <int QP, int QC, typename S>
int launch_batch_stage_s(const DevParams& p, int stage, cudaStream_t s) {
  switch (p.variant) {
    case 1: return launch_batch_stage_v<QP, QC, S, 1>(p, stage, s);
    case 2: return launch_batch_stage_v<QP, QC, S, 2>(p, stage, s);
    default: return launch_batch_stage_v<QP, QC, S, 0>(p, stage, s);
  }
}

template <int QP, int QC>
int launch_batch_stage_t(const DevParams& p, int stage, cudaStream_t s) {
  return p.precision == 1 ? launch_mixed_batch_stage(p, stage, s)
                          : launch_batch_stage_s<QP, QC, double>(p, stage, s);
}

template <int QP, int QC>
int launch_batch_init_t(const DevParams& p, cudaStream_t s) {
  const int nt = 128;
  const int64_t nb = (p.N + nt - 1) / nt;
  if (p.precision == 1) batch_init_kernel<QP, QC, float><<<(unsigned)nb, nt, 0, s>>>(p);
  else batch_init_kernel<QP, QC, double><<<(unsigned)nb, nt, 0, s>>>(p);
  return (int)cudaGetLastError();
}

}  // namespace

bool supported_lattice(int d, int Qp, int Qc) {
#define X(D_, P_, C_) \
  if (d == D_ && Qp == P_ && Qc == C_) return true;
  FDLB_LATTICES(X)
#undef X
  return false;
}

int launch_stage(const DevParams& p, int stage, cudaStream_t s) {
#define X(D_, P_, C_) \
  if (p.d == D_ && p.Qp == P_ && p.Qc == C_) return launch_stage_t<D_, P_, C_>(p, stage, s);
  FDLB_LATTICES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int launch_init_riemann(const DevParams& p, const double* states, int nq, double sx, double sy,
                        cudaStream_t s) {
  RiemannArgs a{};
  const int w = p.d + 2;
  for (int q = 0; q < nq && q < 4; ++q)
    for (int j = 0; j < w; ++j) a.st[q][j] = states[q * w + j];
  a.nq = nq;
  a.sx = sx;
  a.sy = sy;
#define X(D_, P_, C_) \
  if (p.d == D_ && p.Qp == P_ && p.Qc == C_) return launch_init_t<D_, P_, C_>(p, a, s);
  FDLB_LATTICES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int launch_moments(const DevParams& p, double* n, double* ux, double* uy, double* T,
                   cudaStream_t s) {
#define X(D_, P_, C_) \
  if (p.d == D_ && p.Qp == P_ && p.Qc == C_) return launch_moments_t<D_, P_, C_>(p, n, ux, uy, T, s);
  FDLB_LATTICES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int launch_moments_adjoint(const DevParams& p, const double* nbar, const double* uxbar,
                           const double* uybar, const double* Tbar, double* Fbar, cudaStream_t s) {
  const int nt = 128;
  const unsigned nb = (unsigned)((p.N + nt - 1) / nt);
#define X(D_, P_, C_)                                                                       \
  if (p.d == D_ && p.Qp == P_ && p.Qc == C_) {                                              \
    moments_adjoint_kernel<D_, P_, C_><<<nb, nt, 0, s>>>(p, nbar, uxbar, uybar, Tbar, Fbar); \
    return (int)cudaGetLastError();                                                         \
  }
  FDLB_LATTICES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int batch_tile_cells(int variant) {
  switch (variant) {
    case 1: return TileCfg<1, 1>::TX;
    case 2: return TileCfg<1, 2>::TX;
    default: return TileCfg<1, 0>::TX;
  }
}

int launch_batch_stage(const DevParams& p, int stage, cudaStream_t s) {
#define X(P_, C_) \
  if (p.Qp == P_ && p.Qc == C_) return launch_batch_stage_t<P_, C_>(p, stage, s);
  FDLB_BATCH_LATTICES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int launch_batch_init(const DevParams& p, cudaStream_t s) {
#define X(P_, C_) \
  if (p.Qp == P_ && p.Qc == C_) return launch_batch_init_t<P_, C_>(p, s);
  FDLB_BATCH_LATTICES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

}  // namespace fdlb
