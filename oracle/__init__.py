"""FP64 CPU oracle for BP4M decoding on the decoding graph.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py` may import or run anything in this package.  It shares no code, table
or constant generator with the CUDA library: it is a second, deliberately plain
implementation written from the paper, used to check the library.

Modules (each cites the passage it follows):
  philox    Philox4x32-10 counter-based generator (published definition).
  surface   rotated surface code geometry and code-capacity decoding graphs
            (Sec. "MWPM on the surface code").
  circuit   rotated memory-Z circuit and its Z-part detector error model by backward
            Pauli-frame propagation (Sec. "Numerical Results").
  graph     shortest-path weights, observable parities and prior LLRs
            (Eq. two-syn var factors, Eq. priorllr).
  sampler   error sampling and syndrome extraction.
  bp        log-domain sum-product BP, marginalization, convergence check and forced
            convergence (Secs. "Belief Propagation", "Checking convergence",
            "Forced convergence").
  decoders  BP4M (full-T and early-exit), BP4MF, Memory-BP4MF (Sec. "Results").
  brute     exact marginals / MAP by enumerating the valid configurations of Eq. (prob fg).

Parity status: every function here is pinned by a `-m "not gpu"` test under tests/
against values the paper prints, closed forms, brute force or an independent library.
"""
