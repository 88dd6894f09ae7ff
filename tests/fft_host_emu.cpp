// Host run of the device 2-D FFT of csrc/fft.cuh (fft2_forward / fft2_inverse), for the CPU tests: the
// header compiled by the host compiler, one std::thread per CUDA thread of the tile, one shared buffer,
// __syncthreads as a std::barrier over the tile's threads. The line-internal swaps' __syncwarp becomes
// the same barrier: every thread of the tile reaches each of them in the same order, and a barrier
// over the whole tile orders at least what the warp barrier orders on the device.
// Usage: fft_host_emu M V      -> prints "forward <rel L2>  roundtrip <rel L2>" against a direct 2-D DFT in
// double precision (COL layout out of the forward transform, ROW layout back from the inverse).
//        fft_host_emu line BL  -> the same for one BL-point line of the staged passes (line_fft of
// big_line.cuh on 16 threads; frequencies by line_freq).
#include <barrier>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <thread>
#include <vector>

static std::barrier<>* g_bar;
#define __syncthreads() g_bar->arrive_and_wait()
#define __syncwarp() g_bar->arrive_and_wait()
#include "big_line.cuh"
#include "fft.cuh"

using namespace ptycho;
using cd = std::complex<double>;

template <int M, int V>
static int run() {
  using TL = Tile<M>;
  constexpr int E = TL::E, G = TL::G, TR = TL::T / V;
  std::mt19937 rng(M * 10 + V);
  std::normal_distribution<double> nd;
  std::vector<cd> A(M * M);
  for (auto& z : A) z = cd(nd(rng), nd(rng));
  auto W = [](long e) {
    const double t = -2.0 * M_PI * (double)(((e % M) + M) % M) / M;
    return cd(std::cos(t), std::sin(t));
  };
  std::vector<float2> sm(TL::SMEM), tw(G * TL::LDW);
  for (int t = 0; t < G; ++t)
    for (int k = 0; k < TL::LDW; ++k) {
      const cd w = k < E ? W((long)t * k) : cd(0, 0);
      tw[t * TL::LDW + k] = make_float2((float)w.real(), (float)w.imag());
    }
  std::vector<cd> F(M * M), B(M * M);
  std::barrier<> bar(TR);
  g_bar = &bar;
  std::vector<std::thread> th;
  for (int tid = 0; tid < TR; ++tid)
    th.emplace_back([&, tid] {
      float2 a[V][E];
      for (int v = 0; v < V; ++v) {
        const int vt = tid + v * TR, line = vt / G, t = vt % G;
        for (int j = 0; j < E; ++j) {
          const cd z = A[line * M + t + G * j];
          a[v][j] = make_float2((float)z.real(), (float)z.imag());
        }
      }
      fft2_forward<M, V>(a, sm.data(), tw.data(), tid);
      for (int v = 0; v < V; ++v) {
        const int vt = tid + v * TR, c = vt / G, t = vt % G;
        for (int r = 0; r < E; ++r) F[col_freq<M>(t, r) * M + c] = cd(a[v][r].x, a[v][r].y);
      }
      fft2_inverse<M, V>(a, sm.data(), tw.data(), tid);
      for (int v = 0; v < V; ++v) {
        const int vt = tid + v * TR, line = vt / G, t = vt % G;
        for (int j = 0; j < E; ++j) B[line * M + t + G * j] = cd(a[v][j].x, a[v][j].y);
      }
    });
  for (auto& t : th) t.join();
  // direct 2-D DFT (rows, then columns) in double
  std::vector<cd> R(M * M), Y(M * M);
  for (int y = 0; y < M; ++y)
    for (int v = 0; v < M; ++v) {
      cd s = 0;
      for (int x = 0; x < M; ++x) s += A[y * M + x] * W((long)v * x);
      R[y * M + v] = s;
    }
  for (int u = 0; u < M; ++u)
    for (int v = 0; v < M; ++v) {
      cd s = 0;
      for (int y = 0; y < M; ++y) s += R[y * M + v] * W((long)u * y);
      Y[u * M + v] = s;
    }
  double e1 = 0, n1 = 0, e2 = 0, n2 = 0;
  for (int i = 0; i < M * M; ++i) {
    e1 += std::norm(F[i] - Y[i]);
    n1 += std::norm(Y[i]);
    e2 += std::norm(B[i] / (double)(M * M) - A[i]);
    n2 += std::norm(A[i]);
  }
  std::printf("forward %.3e roundtrip %.3e\n", std::sqrt(e1 / n1), std::sqrt(e2 / n2));
  return 0;
}

template <int BL>
static int run_line() {
  using BS_ = BigShape<BL>;
  constexpr int E = BS_::E;
  std::mt19937 rng(BL);
  std::normal_distribution<double> nd;
  std::vector<cd> x(BL);
  for (auto& z : x) z = cd(nd(rng), nd(rng));
  auto W = [](long e) {
    const double t = -2.0 * M_PI * (double)(((e % BL) + BL) % BL) / BL;
    return cd(std::cos(t), std::sin(t));
  };
  std::vector<float2> sw(BS_::SWN), tw(BS_::TWN);
  for (int i = 0; i < BS_::TWN; ++i) {  // as load_tw: W_BL^(t k2) for k2 < E, zero beyond
    const int t = i / BS_::TWS, k2 = i % BS_::TWS;
    const cd w = k2 < E ? W((long)t * k2) : cd(0, 0);
    tw[i] = make_float2((float)w.real(), (float)w.imag());
  }
  std::vector<cd> F(BL), B(BL);
  std::barrier<> bar(BT);
  g_bar = &bar;
  std::vector<std::thread> th;
  for (int t = 0; t < BT; ++t)
    th.emplace_back([&, t] {
      float2 a[E];
      for (int j = 0; j < E; ++j) a[j] = make_float2((float)x[t + 16 * j].real(), (float)x[t + 16 * j].imag());
      line_fft<BL, false>(a, sw.data(), tw.data(), t);
      for (int r = 0; r < E; ++r) F[line_freq<BL>(t, r)] = cd(a[r].x, a[r].y);
      line_fft<BL, true>(a, sw.data(), tw.data(), t);
      for (int j = 0; j < E; ++j) B[t + 16 * j] = cd(a[j].x, a[j].y);
    });
  for (auto& t : th) t.join();
  double e1 = 0, n1 = 0, e2 = 0, n2 = 0;
  for (int k = 0; k < BL; ++k) {
    cd s = 0;
    for (int n = 0; n < BL; ++n) s += x[n] * W((long)k * n);
    e1 += std::norm(F[k] - s);
    n1 += std::norm(s);
    e2 += std::norm(B[k] / (double)BL - x[k]);
    n2 += std::norm(x[k]);
  }
  std::printf("forward %.3e roundtrip %.3e\n", std::sqrt(e1 / n1), std::sqrt(e2 / n2));
  return 0;
}

int main(int argc, char** argv) {
  if (argc == 3 && std::string(argv[1]) == "line") {
    const int BL = std::atoi(argv[2]);
    return BL == 256 ? run_line<256>() : BL == 512 ? run_line<512>() : 2;
  }
  if (argc != 3) return 2;
  const int M = std::atoi(argv[1]), V = std::atoi(argv[2]);
  if (M == 8 && V == 1) return run<8, 1>();
  if (M == 16 && V == 1) return run<16, 1>();
  if (M == 32 && V == 1) return run<32, 1>();
  if (M == 64 && V == 1) return run<64, 1>();
  if (M == 64 && V == 2) return run<64, 2>();
  if (M == 128 && V == 2) return run<128, 2>();
  if (M == 128 && V == 4) return run<128, 4>();
  return 2;
}
