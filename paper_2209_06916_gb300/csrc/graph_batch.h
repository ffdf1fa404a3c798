// One CUDA graph for a batch of graph-resident solves (internal to the
// library; driver.cu implements it, serve.cu uses it).  Each solve is an
// independent branch of the graph: its prologue, stop-test init and
// conditional while node, so one launch runs the whole batch and the graph
// executor overlaps the branches.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mgrit.h"

// Capture every solve of hs into one graph and instantiate it.
int batch_graph_build(mgrit_handle* const* hs, int64_t n, cudaGraphExec_t* out);
// Initial iterates (u0s[i]: host or device, nx_i values) and device states,
// one launch of the batch graph, the states back; synchronises st.
int batch_graph_run(mgrit_handle* const* hs, int64_t n, const double* const* u0s, cudaGraphExec_t ge,
                    cudaStream_t st);
// Statistics of solve h after batch_graph_run; returns its status.
int batch_graph_stats(const mgrit_handle* h, mgrit_stats* stats);
// Measured geometry tuning on (default) or off for the calling thread.
void set_measured_tuning(bool on);
// Build a handle's graph-resident solve now (mgrit_solve_async then only
// launches it).
int solve_graph_prepare(mgrit_handle* h);
// mgrit_setup and solve-graph capture without waiting for the device, for
// the calling thread (default off).
void set_setup_nowait(bool on);
// Queue the initial condition u0 (device or pinned host memory: nothing
// waits) for the next mgrit_solve_async(h, NULL).
extern "C" __attribute__((visibility("hidden"))) int solve_stage_initial(mgrit_handle* h, const double* u0);
