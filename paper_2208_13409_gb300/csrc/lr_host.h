// lr_host.h -- host-side helpers shared by the single-simulation API
// (lr_api.cu) and the batch API (lr_batch.cu).
#pragma once
#include "../../include/lr.h"
#include "lr_dev.cuh"
#include <stddef.h>

// Validate a configuration; on failure write the reason to why.
bool lr_config_ok(const lr_config* c, char* why, size_t nwhy);
// Grid constants of a configuration (materials, offsets and slot left as they are).
void lr_fill_grid(const lr_config& f, LrGrid& g);
// Field `field` (LR_F_*) of one simulation as doubles into device memory dst;
// s is its current state, prev the other half of its double buffer, rows a
// device scratch of 8 (ny + 1) doubles.  *unknown is set for an unknown field.
cudaError_t lr_field_view(const LrGrid& g, const LrState& s, const LrState& prev, const LrWork& w, double* rows,
                          int field, double* dst, cudaStream_t st, bool* unknown);
// Number of doubles of a field, 0 if unknown.
size_t lr_field_count(const LrGrid& g, int field);
// The auxiliary stream of the interface kernels, at the device's highest
// priority: its blocks are scheduled ahead of the step kernels they run
// beside, so the short, latency-bound interface work is not left to the
// tail of lr_mat_flux.
cudaError_t lr_create_aux_stream(cudaStream_t* s);
