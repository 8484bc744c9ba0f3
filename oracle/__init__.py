"""FP64 CPU oracle for MN-BaB bounding (Ferrari et al., ICLR 2022).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: it exists so that tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` can check and time the GPU library
against a plain, slow, obviously correct restatement of the method.  It
shares no code with the CUDA path; both read their inputs from ``synth``.

Modules
-------
``core``   networks, back-substitution through affine and ReLU layers (Sec. 3.1,
           affine and ReLU back-substitution equations), concretisation over the
           input box (Eq. minimum), the counterexample candidate (Sec. 3.1, upper
           bounding), intermediate bounds, projected Adam (Sec. 3.1) and ACS
           branching scores (Sec. 3.2).
``mnc``    multi-neuron constraint generator over k=3 neuron groups (the paper
           defers to PRIMA; the construction here is this project's reading).
``bab``    branch-and-bound driver (Sec. 2.2, Sec. 3.2 enforcing splits).
``exact``  exact minima of tiny networks by activation-pattern enumeration
           with one LP per pattern (used only to pin the rest).

Parity status of each function is given in its docstring.  Pieces whose
values the paper does not fix (Adam hyper-parameters, FIFO queue order, the
group policy of the constraint generator, the eps calibration) are
"parity unpinned": they are self-consistent definitions of this project.
"""
