// Runtime-N dispatch of the templated stage kernel.
#pragma once
#include "bb_stage.cuh"
#include "bb_stage_warp.cuh"
#include "bb_pipe.cuh"
#include "bb_stage_thread.cuh"

#define BBDG_INSTANTIATE_STAGE(T)                                                              \
  namespace bbdg {                                                                             \
  template <>                                                                                  \
  int launch_bb_stage<T>(int N, const StageArgs<T>& a, int64_t S, cudaStream_t st,             \
                         size_t* smem) {                                                       \
    switch (N) {                                                                               \
      case 1: return launch_bb_stage_n<T, 1>(a, S, st, smem);                                  \
      case 2: return launch_bb_stage_n<T, 2>(a, S, st, smem);                                  \
      case 3: return launch_bb_stage_n<T, 3>(a, S, st, smem);                                  \
      case 4: return launch_bb_stage_n<T, 4>(a, S, st, smem);                                  \
      case 5: return launch_bb_stage_n<T, 5>(a, S, st, smem);                                  \
      case 6: return launch_bb_stage_n<T, 6>(a, S, st, smem);                                  \
      case 7: return launch_bb_stage_n<T, 7>(a, S, st, smem);                                  \
      case 8: return launch_bb_stage_n<T, 8>(a, S, st, smem);                                  \
      case 9: return launch_bb_stage_n<T, 9>(a, S, st, smem);                                  \
      case 10: return launch_bb_stage_n<T, 10>(a, S, st, smem);                                \
      default: return BBDG_EUNSUPPORTED;                                                       \
    }                                                                                          \
  }                                                                                            \
  size_t bb_stage_smem_t_##T(int N, int E, int lv) {                                           \
    switch (N) {                                                                               \
      case 1: return bb_smem_bytes_t<T, 1>(E, lv);                                             \
      case 2: return bb_smem_bytes_t<T, 2>(E, lv);                                             \
      case 3: return bb_smem_bytes_t<T, 3>(E, lv);                                             \
      case 4: return bb_smem_bytes_t<T, 4>(E, lv);                                             \
      case 5: return bb_smem_bytes_t<T, 5>(E, lv);                                             \
      case 6: return bb_smem_bytes_t<T, 6>(E, lv);                                             \
      case 7: return bb_smem_bytes_t<T, 7>(E, lv);                                             \
      case 8: return bb_smem_bytes_t<T, 8>(E, lv);                                             \
      case 9: return bb_smem_bytes_t<T, 9>(E, lv);                                             \
      case 10: return bb_smem_bytes_t<T, 10>(E, lv);                                           \
      default: return 0;                                                                       \
    }                                                                                          \
  }                                                                                            \
  template <>                                                                                  \
  int launch_bb_warp<T>(int N, const StageArgs<T>& a, int64_t S, int W, cudaStream_t st) {     \
    switch (N) {                                                                               \
      case 1: return launch_bb_warp_n<T, 1>(a, S, W, st);                                      \
      case 2: return launch_bb_warp_n<T, 2>(a, S, W, st);                                      \
      case 3: return launch_bb_warp_n<T, 3>(a, S, W, st);                                      \
      case 4: return launch_bb_warp_n<T, 4>(a, S, W, st);                                      \
      case 5: return launch_bb_warp_n<T, 5>(a, S, W, st);                                      \
      case 6: return launch_bb_warp_n<T, 6>(a, S, W, st);                                      \
      case 7: return launch_bb_warp_n<T, 7>(a, S, W, st);                                      \
      case 8: return launch_bb_warp_n<T, 8>(a, S, W, st);                                      \
      case 9: return launch_bb_warp_n<T, 9>(a, S, W, st);                                      \
      case 10: return launch_bb_warp_n<T, 10>(a, S, W, st);                                    \
      default: return BBDG_EUNSUPPORTED;                                                       \
    }                                                                                          \
  }                                                                                            \
  size_t bb_warp_smem_t_##T(int N, int W) {                                                    \
    switch (N) {                                                                               \
      case 1: return warp_smem_bytes_t<T, 1>(W);                                               \
      case 2: return warp_smem_bytes_t<T, 2>(W);                                               \
      case 3: return warp_smem_bytes_t<T, 3>(W);                                               \
      case 4: return warp_smem_bytes_t<T, 4>(W);                                               \
      case 5: return warp_smem_bytes_t<T, 5>(W);                                               \
      case 6: return warp_smem_bytes_t<T, 6>(W);                                               \
      case 7: return warp_smem_bytes_t<T, 7>(W);                                               \
      case 8: return warp_smem_bytes_t<T, 8>(W);                                               \
      case 9: return warp_smem_bytes_t<T, 9>(W);                                               \
      case 10: return warp_smem_bytes_t<T, 10>(W);                                             \
      default: return 0;                                                                       \
    }                                                                                          \
  }                                                                                            \
  template <>                                                                                  \
  int launch_bb_pipe<T>(int N, const StageArgs<T>& a, int64_t S, cudaStream_t st) {            \
    switch (N) {                                                                               \
      case 1: return launch_bb_pipe_n<T, 1>(a, S, st);                                         \
      case 2: return launch_bb_pipe_n<T, 2>(a, S, st);                                         \
      case 3: return launch_bb_pipe_n<T, 3>(a, S, st);                                         \
      case 4: return launch_bb_pipe_n<T, 4>(a, S, st);                                         \
      case 5: return launch_bb_pipe_n<T, 5>(a, S, st);                                         \
      case 6: return launch_bb_pipe_n<T, 6>(a, S, st);                                         \
      case 7: return launch_bb_pipe_n<T, 7>(a, S, st);                                         \
      case 8: return launch_bb_pipe_n<T, 8>(a, S, st);                                         \
      case 9: return launch_bb_pipe_n<T, 9>(a, S, st);                                         \
      case 10: return launch_bb_pipe_n<T, 10>(a, S, st);                                       \
      default: return BBDG_EUNSUPPORTED;                                                       \
    }                                                                                          \
  }                                                                                            \
  size_t bb_pipe_smem_t_##T(int N) {                                                           \
    switch (N) {                                                                               \
      case 1: return pipe_smem_bytes_t<T, 1>();                                                \
      case 2: return pipe_smem_bytes_t<T, 2>();                                                \
      case 3: return pipe_smem_bytes_t<T, 3>();                                                \
      case 4: return pipe_smem_bytes_t<T, 4>();                                                \
      case 5: return pipe_smem_bytes_t<T, 5>();                                                \
      case 6: return pipe_smem_bytes_t<T, 6>();                                                \
      case 7: return pipe_smem_bytes_t<T, 7>();                                                \
      case 8: return pipe_smem_bytes_t<T, 8>();                                                \
      case 9: return pipe_smem_bytes_t<T, 9>();                                                \
      case 10: return pipe_smem_bytes_t<T, 10>();                                              \
      default: return 0;                                                                       \
    }                                                                                          \
  }                                                                                            \
  template <>                                                                                  \
  int launch_bb_thread<T>(int N, const StageArgs<T>& a, int64_t S, cudaStream_t st) {          \
    switch (N) {                                                                               \
      case 1: return launch_bb_thread_n<T, 1>(a, S, st);                                       \
      case 2: return launch_bb_thread_n<T, 2>(a, S, st);                                       \
      default: return BBDG_EUNSUPPORTED;                                                       \
    }                                                                                          \
  }                                                                                            \
  template <>                                                                                  \
  int launch_receivers<T>(int N, const T* q, T* traces, int64_t S, int64_t K, int nrec,        \
                          const int32_t* elem, const T* basis, cudaStream_t st) {              \
    if (nrec <= 0 || S <= 0) return BBDG_OK;                                                   \
    dim3 grid((unsigned)((nrec * 32 + 255) / 256), (unsigned)S);                               \
    receiver_kernel<T><<<grid, 256, 0, st>>>(q, traces, K, np_of(N), nrec, elem, basis);       \
    return cudaGetLastError() == cudaSuccess ? BBDG_OK : BBDG_ECUDA;                           \
  }                                                                                            \
  }
