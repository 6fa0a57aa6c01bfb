"""CPU oracle for the RLWE-PIR first-dimension scan.  Test infrastructure only:
the product path never imports this package."""
