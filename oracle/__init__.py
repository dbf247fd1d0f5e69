"""CPU oracle for the amplitude-damped bucket-brigade QRAM trajectory method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_2609_34935_b300``) and never imports it.

Parts:
  - ``qram_oracle.c`` (loaded through ``oracle.core``): plain full evolution
    of every branch of every trajectory over the sparse dictionary of App. A,
    Eq. (27), with the joint damping sampler of Sec. IV.D; the classifier of
    Eq. (7) / Eq. (9); Philox4x32-10.
  - ``oracle.closed_forms``: the closed forms of Prop. 1, Lemma 1,
    Theorems 1-2, Eqs. (13)-(16), (22)-(24), written out directly.
  - ``oracle.dm``: a brute-force density-matrix simulation of the whole
    loading circuit (App. C) for n <= 2.
"""
