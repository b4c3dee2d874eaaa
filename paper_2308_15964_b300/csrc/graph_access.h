// Read-only view of a built graph's host arrays, for the server (which
// copies a graph into its device pools).  Internal to the library.
#pragma once

#include <stddef.h>

#include "spx.h"
#include "spx_internal.h"

namespace spx {

struct GraphView {
  const TaskDesc* tasks;
  size_t ntasks;
  const TileDesc* tiles;
  size_t ntiles;
  const CUtensorMap* maps;
  size_t nmaps;
  const uint32_t* rec_handle;
  const uint32_t* rec_seq;
  const uint8_t* rec_mode;
  size_t nrec;
  const uint32_t* task_rec;  // ntasks + 1 entries
  unsigned long long cand_edges;
  unsigned long long items;  // queue entries of all phases of all tasks
};

}  // namespace spx

// SPX_ERR_STATE if the graph is running; SPX_ERR_INVALID_ARG if NULL.
int spx_graph_view(spx_graph_t g, spx::GraphView* v);
