"""Select-join-group-by queries over a star schema resident in HBM (Section 5.3).

A query (plain dict: fact predicates, joins with dimension filters and an optional
group attribute per dimension, one SUM expression) compiles to one of two plan shapes:

* ``mode="filtered"`` — the paper's plan: one build kernel per joined dimension with the
  dimension filter applied at build time and the group attribute as the table value,
  then one fused probe kernel over the fact table.  Tables are sized from the filter's
  expected selectivity with an 8-sigma margin; a full table is flagged on the device and
  ``check_device_errors`` raises, so a wrong estimate never goes unnoticed.
* ``mode="resident"`` — every dimension has one resident table, built when the schema is
  loaded (a direct table: the slot of key k is k, the paper's "perfect hashing" of dense
  dimension keys, so the four tables total about 37 MB and stay in L2), whose value packs
  all of the dimension's attribute codes into bit fields; a query's dimension filters and
  group attribute become bit-field predicates and a bit-field group code on that shared
  table, so a query needs no build at all.  A shared scan of such queries tags every
  dimension row with the bitmap of the batch's queries it satisfies and reads one tag
  per dimension and fact row (``crys_run_plans_tagged``).

Both shapes give identical results (integer sums and counts per group).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import torch

from . import (HashTable, crys_get_tile, crys_hash_build, crys_hash_init, crys_pack_fields, crys_run_plan,
               crys_run_plans_tagged, crys_run_plans_tagged_bytes, crys_tagged_block_bytes,
               crys_tagged_launch, crys_tagged_prepare, make_plan, make_table, capacity_for,
               ACCUMULATE, MAX_PLANS, HASH_DIRECT, HASH_IDENT, OK, OP_TAGGED_SCAN, TAG_ANNOTATE)


@dataclass
class Schema:
    """Names and domains of the fact columns and of each dimension's attributes.

    The package knows no particular workload: whoever loads a star schema states its
    column names, each dimension's foreign-key column and attribute cardinalities (the
    dictionary-encoded domains of Section 5.2), e.g. ``Schema.from_spec(cols, dims)``."""
    fact_cols: list
    dims: dict          # dim -> {"fk": fact col name, "attrs": {attr: cardinality}}

    @classmethod
    def from_spec(cls, fact_cols, dims: dict) -> "Schema":
        """From a column list and a {dim: {"fk": col, "attrs": {attr: card}, ...}} mapping
        (other keys of a dimension's entry are ignored)."""
        return cls(list(fact_cols), {d: {"fk": s["fk"], "attrs": dict(s["attrs"])} for d, s in dims.items()})


@dataclass
class CompiledQuery:
    query: dict
    plan: object                       # crys_plan
    sums: torch.Tensor
    counts: torch.Tensor
    tables: list = field(default_factory=list)   # per-query HashTables kept alive with the plan
    groups: int = 1
    serial: int = field(default_factory=itertools.count().__next__)   # unique per compiled plan

    @property
    def table_bytes(self) -> int:
        return sum(t.nbytes for t in self.tables)

    @property
    def output_bytes(self) -> int:
        return 16 * self.groups


class ResidentStarSchema:
    """Fact and dimension columns (and the packed dimension tables) resident on one device."""

    def __init__(self, schema: Schema, fact: dict, dims: dict, stream=None):
        self.schema = schema
        self.fact = fact
        self.dims = dims
        self.cols = [fact[c] for c in schema.fact_cols]
        self.table = make_table(self.cols)
        self.n_rows = self.cols[0].numel()
        self.device = self.cols[0].device
        self.fields = {}     # dim -> {attr: (shift, bits)}
        self.resident = {}   # dim -> HashTable(key -> packed attribute codes)
        self.packed = {}
        for d, spec in schema.dims.items():
            shift, fields = 0, {}
            for attr, card in spec["attrs"].items():
                bits = max(1, int(card - 1).bit_length())
                fields[attr] = (shift, bits)
                shift += bits
            if shift > 31:
                raise ValueError(f"attributes of {d} need {shift} bits")
            dim = dims[d]
            rows = dim["key"].numel()
            names = list(fields)
            packed = torch.empty(rows, dtype=torch.int32, device=self.device)
            crys_pack_fields([dim[a] for a in names], [fields[a][0] for a in names],
                             [fields[a][1] for a in names], rows, packed, stream)
            self.fields[d] = fields
            self.packed[d] = packed
            # Dimension keys are dense (0..rows-1, shuffled), so the resident table is a
            # direct table: slot k holds key k.  Other key sets fall back to identity
            # hashing with linear probing.
            keys = dim["key"]
            lo, hi = (int(keys.min().item()), int(keys.max().item())) if rows else (0, 0)
            if rows and lo >= 0 and hi < (1 << 31):
                self.resident[d] = HashTable.build(keys, packed, capacity=hi + 1, stream=stream,
                                                   kind=HASH_DIRECT)
            else:
                self.resident[d] = HashTable.build(keys, packed, stream=stream, kind=HASH_IDENT)
        # query bitmaps of the latest shared scan: one 8-byte entry per slot of each
        # (fact column, table) pair; each resident table is joined through one column
        need = sum((t.capacity * 8 + 15) // 16 * 16 for t in self.resident.values())
        self._scratch = torch.empty(max(need, 16), dtype=torch.uint8, device=self.device)

    @property
    def resident_bytes(self) -> int:
        return sum(t.nbytes for t in self.resident.values())

    # -- sizing -------------------------------------------------------------------
    def expected_rows(self, join: dict) -> float:
        d = join["dim"]
        rows = self.dims[d]["key"].numel()
        sel = 1.0
        for attr, lo, hi in join["filters"]:
            sel *= (hi - lo + 1) / self.schema.dims[d]["attrs"][attr]
        return rows * sel

    def table_capacity(self, join: dict) -> int:
        mean = self.expected_rows(join)
        bound = mean + 8.0 * math.sqrt(mean) + 64
        rows = self.dims[join["dim"]]["key"].numel()
        return capacity_for(int(min(rows, bound)))

    def groups(self, query: dict) -> int:
        g = 1
        for j in query["joins"]:
            if j["group"] is not None:
                g *= self.schema.dims[j["dim"]]["attrs"][j["group"]]
        return g

    def memory_needed(self, query: dict, mode: str = "resident") -> int:
        """Device bytes a query holds while admitted: its own hash tables (none with the
        resident tables) and its outputs (sums and counts, 16 B per group)."""
        tb = 0 if mode == "resident" else sum(8 * self.table_capacity(j) for j in query["joins"])
        return tb + 16 * self.groups(query)

    # -- compilation ----------------------------------------------------------------
    def compile(self, query: dict, mode: str = "resident", stream=None, zero: bool = True) -> CompiledQuery:
        """Plan of one query; with zero=False its outputs are left uninitialised (a
        replayed scan clears them in the query's first launch)."""
        names = self.schema.fact_cols
        preds = [(names.index(c), lo, hi) for (c, lo, hi) in query["fact_preds"]]
        joins, tables = [], []
        for j in query["joins"]:
            d = j["dim"]
            spec = self.schema.dims[d]
            fk = names.index(spec["fk"])
            card = spec["attrs"][j["group"]] if j["group"] is not None else 0
            if mode == "resident":
                fields = self.fields[d]
                gfield = fields[j["group"]] if j["group"] is not None else (0, 0)
                fpreds = [(fields[a][0], fields[a][1], lo, hi) for (a, lo, hi) in j["filters"]]
                joins.append((fk, self.resident[d], card, gfield, fpreds))
            elif mode == "filtered":
                dim = self.dims[d]
                ht = HashTable(self.table_capacity(j), self.device)
                crys_hash_init(ht.struct, stream)
                filters = [(dim[a], lo, hi) for (a, lo, hi) in j["filters"]]
                vals = dim[j["group"]] if j["group"] is not None else None
                crys_hash_build(dim["key"], vals, dim["key"].numel(), filters, ht.struct, stream)
                joins.append((fk, ht, card))
                tables.append(ht)
            else:
                raise ValueError(f"unknown mode {mode}")
        op, a, b = query["agg"]
        agg = (op, names.index(a), names.index(b) if b is not None else None)
        g = self.groups(query)
        alloc = torch.zeros if zero else torch.empty
        sums = alloc(g, dtype=torch.int64, device=self.device)
        counts = alloc(g, dtype=torch.int64, device=self.device)
        plan = make_plan(preds, joins, agg, sums, counts)
        return CompiledQuery(query, plan, sums, counts, tables, g)

    # -- execution ------------------------------------------------------------------
    def run(self, cq: CompiledQuery, stream=None) -> None:
        """One query, one fused probe kernel over all fact rows."""
        crys_run_plan(self.table, cq.plan, stream)

    def scratch(self, need: int) -> torch.Tensor:
        """The query-bitmap scratch, grown when a batch needs more.  Earlier launches on
        any stream may still read or write the old block, so the device is drained before
        it goes back to the allocator (growth is rare: the store is built with room for
        every resident table)."""
        if self._scratch.numel() < need:
            torch.cuda.synchronize(self.device)
            self._scratch = None
            self._scratch = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self._scratch

    def run_shared(self, cqs: list, row_begin: int = 0, row_end: int | None = None,
                   accumulate: bool = False, stream=None) -> None:
        """Up to 32 queries in one shared scan over rows [row_begin, row_end); with the
        resident direct tables the batch is tagged with query bitmaps."""
        if len(cqs) > MAX_PLANS:
            raise ValueError("at most 32 queries per shared scan")
        row_end = self.n_rows if row_end is None else row_end
        plans = [c.plan for c in cqs]
        need = crys_run_plans_tagged_bytes(self.table, plans)
        scratch = self.scratch(need) if need else None
        crys_run_plans_tagged(self.table, plans, row_begin, row_end, ACCUMULATE if accumulate else 0,
                              scratch, scratch.numel() if need else 0, stream)

    def query_columns(self, query: dict) -> set:
        cols = {c for (c, _, _) in query["fact_preds"]}
        cols |= {self.schema.dims[j["dim"]]["fk"] for j in query["joins"]}
        op, a, b = query["agg"]
        cols.add(a)
        if b is not None:
            cols.add(b)
        return cols

    def bytes_scanned(self, query: dict) -> int:
        """Algorithmic bytes of one query: each fact column it reads, once (4 B/row)."""
        return 4 * self.n_rows * len(self.query_columns(query))


class ReplayedScan:
    """Tagged shared scans of a serving loop through captured CUDA graphs.

    A launch's arguments go to a pinned host block (``crys_tagged_prepare``); the graph
    replays {copy of the block to the device, ``crys_tagged_launch``}.  Two pinned blocks
    alternate, each with its own graph, so the host prepares launch k+1 while launch k
    runs; a block is rewritten only after the replay that read it has finished."""

    def __init__(self, store: ResidentStarSchema, stream: torch.cuda.Stream):
        self.store = store
        self.stream = stream
        nb = crys_tagged_block_bytes()
        self.block_bytes = nb                # bytes copied host -> device per launch
        self.dev_block = torch.empty(nb, dtype=torch.uint8, device=store.device)
        self.host = [torch.empty(nb, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        self.graphs = [None, None]
        self.shape = None    # tile shape the graphs were captured with
        self.done = [None, None]
        self.k = 0
        self.replays = 0
        self._batch = None

    def _capture(self, i: int) -> None:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.dev_block.copy_(self.host[i], non_blocking=True)
            crys_tagged_launch(self.dev_block)
        self.graphs[i] = g

    def launch(self, cqs: list, row_begin: int, row_end: int, zero: list) -> bool:
        """One launch of `cqs` over rows [row_begin, row_end), adding to their outputs
        after clearing those of the plans listed in `zero`; False when the batch cannot
        use the replayed launch (nothing was enqueued)."""
        plans = [c.plan for c in cqs]
        need = crys_run_plans_tagged_bytes(self.store.table, plans)
        if not need:
            return False
        scratch = self.store.scratch(need)
        batch = (tuple(c.serial for c in cqs), scratch.data_ptr())
        i = self.k % 2
        if self.done[i] is not None:
            self.done[i].synchronize()
        flags = TAG_ANNOTATE if batch != self._batch else 0
        rc = crys_tagged_prepare(self.store.table, plans, row_begin, row_end, flags, list(zero), scratch,
                                 scratch.numel(), self.host[i].data_ptr())
        if rc != OK:
            return False
        shape = crys_get_tile(OP_TAGGED_SCAN)
        if shape != self.shape:                 # a new tile shape: capture both graphs again
            for j in range(2):
                if self.done[j] is not None:
                    self.done[j].synchronize()
            self.graphs = [None, None]
            self.shape = shape
        if self.graphs[i] is None:
            self._capture(i)
        with torch.cuda.stream(self.stream):
            self.graphs[i].replay()
            ev = torch.cuda.Event()
            ev.record(self.stream)
        self.done[i] = ev
        self._batch = batch
        self.k += 1
        self.replays += 1
        return True
