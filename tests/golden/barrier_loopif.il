; Sec. 6.2: the barrier payoff expression used to show the Futhark backend,
;   loopif(model("AAPL", 0) <= 4000.0, 0.0, 2000.0 * payoff(0,X,Y), t)
; with AAPL = label 0, X = 0, Y = 1 and the window t = template variable $0.
(loopif (le (model 0 0) 4000.0) 0.0 (mult 2000.0 (payoff 0 0 1)) $0)
